// lr.cu -- the encrypted logistic-regression gradient step of a worker
// (Sec. 4: Eq. 5-8 with a Table 2 polynomial; Algorithm 1).
//
// Packing: each data ciphertext holds g samples interleaved, slot g*f + s =
// y_s * x_{s,f}; W holds w_f in slots g*f + s for every s.  Because slot
// rotations are cyclic over all N/2 slots, the sum of the rotations by o*g
// for o < F = N/(2g) leaves in every slot g*f + s the full inner product
// m_s = w . z_s of its own sample, so no mask is needed before the
// polynomial.  After the polynomial, the sum of the rotations by o < g
// collects the per-feature sum on slots = 0 mod g, a 0/1 mask keeps those,
// and the sum of the rotations by -o copies it back to all g slots.  Each
// rotate-and-sum runs in hoisted stages (rotsum_batch) of up to fifteen
// rotations (rotsum_stages).
//
// Op sequence and scale plan (doubles, same order as the CPU oracle; l0 the
// input level, q[i] the limb primes):
//   U  = HMult(Z_k, W)                      sU = sZ*sW/q[l0-1]
//   M  = sum over o < F of rot(U, o*g)       (hoisted stages)
//   T  = HMult(M, M)                        sT = sU*sU/q[l0-2]
//   sS = ((sW*q[l0-5])*q[l0-4]) / (mask_scale*sZ)
//   A  = rescale(M * round(c3*lr*sigA)),    sigA = ((sS*q[l0-3])/sT * q[l0-2])/sU
//   C  = HMult(T, A)
//   B  = rescale(M * round(c1*lr*sigB)),    sigB = (sS*q[l0-2])/sU, dropped one level
//   Q  = rescale(T * round(c2*lr*sigQ)),    sigQ = (sS*q[l0-3])/sT   (c2 != 0)
//   S  = C + B (+ Q) + round(c0*lr*scale(C))
//   D  = sum_k tensor(S_k, drop(Z_k)) ;  G = rescale(relinearise(D))   (one key switch per shard)
//   H  = sum over o < g of rot(G, o) ;  R = rescale(H (x) mask) ;  R <- sum over o < g of rot(R, -o)
//   W' = drop(W) + R                        (scale sW, level l0-5)
//   W' += rescale(drop(W, l0-4) * round(-lr l2 q[l0-5]))   with the L2 regulariser (Eq. 4, 6)
#include <math.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <map>
#include <string>
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
  // stream-ordered: the context's stream may be a non-blocking one, which
  // the legacy default stream's copies do not order against
  HE_CUDA(cudaMemcpyAsync(z, host.data(), sizeof(double) * nh, cudaMemcpyHostToDevice, c->stream));
  HE_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c->stream));
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
  int64_t kR;  // round(-lr l2 q_{l0-5}): the regulariser's constant (0: none)
  bool has_c2;
};

// Scale plan; for inference the polynomial's output S is produced at W's scale
// (it is the result, two levels above the lowest), otherwise at the scale
// that brings the step's output back to W's scale (see the header comment).
static int lr_plan(const he_ctx* c, uint32_t l0, double sZ, double sW, const he_lr_config* cfg, bool infer,
                   LrPlan* p) {
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
  p->sS = infer ? sW : ((sW * (double)q[l0 - 5]) * (double)q[l0 - 4]) / (ms * sZ);
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
  p->kR = 0;
  if (infer) return HE_OK;
  p->sG = p->sC * sZ / (double)q[l0 - 4];
  p->sR = (p->sG * ms) / (double)q[l0 - 5];
  if (!scales_eq(p->sR, sW)) return fail(HE_ESCALE, "output scale mismatch");
  if (cfg->l2 != 0.0) {  // - lr l2 w at W's scale: w times round(-lr l2 q_{l0-5}), rescaled by q_{l0-5}
    if (!to_int(-lr * cfg->l2 * (double)q[l0 - 5], &p->kR)) return fail(HE_EINVAL, "l2 constant beyond int64");
    if (!scales_eq((sW * (double)q[l0 - 5]) / (double)q[l0 - 5], sW)) return fail(HE_ESCALE, "l2 term scale");
  }
  return HE_OK;
}

// Per-ciphertext words of the circuit's intermediates at input level l0:
// U, T, A, C, B, Q, Tmp, and the gathered copies of Z and W.
static size_t lr_ct_words(const he_ctx* c, uint32_t l0) {
  const size_t n = c->n;
  return n * 2 * ((l0 - 1) + (l0 - 2) + (l0 - 2) + (l0 - 3) + (l0 - 2) + (l0 - 3) + (l0 - 1) + 2 * l0) + 9 * 32;
}

// Scratch words of one operation of the step: those of the per-ciphertext
// part over `chunk` ciphertexts and those of the finish over `ns` sums.
static size_t lr_op_words(const he_ctx* c, uint32_t l0, uint32_t chunk, uint32_t ns) {
  size_t w = mul_words(c, l0, chunk, true);
  w = std::max(w, rotsum_words(c, l0 - 1, chunk));
  w = std::max(w, rescale_words(c, l0 - 1, chunk));
  w = std::max(w, rotsum_words(c, l0 - 4, ns));
  w = std::max(w, ks_words(c, l0 - 3, ns) + (size_t)ns * 2 * (l0 - 3) * c->n + rescale_words(c, l0 - 3, ns) + 64);
  w = std::max(w, rescale_words(c, l0 - 4, ns) + (size_t)ns * 2 * (l0 - 4) * c->n);
  return w + 64;
}

// Galois elements of the step's three rotate-and-sums, stage by stage.
struct LrGal {
  std::vector<std::vector<uint64_t>> in, up, down;
};

// The stages of a rotate-and-sum over offsets 0, step, ..., (2^count - 1) step:
// stages of three doublings (rotations by s, 2s, ..., 7s in one hoisted
// stage, then s <- 8s), the first of four when count = 1 mod 3 and a last
// one of two when count = 2 mod 3 (every stage pays one ModUp and one
// ModDown, each rotation one inner product).
static void rotsum_stages(int log_n, int32_t step, uint32_t count, std::vector<std::vector<uint64_t>>* out) {
  std::vector<uint32_t> sizes(count / 3, 3);
  if (count % 3 == 1) {
    if (sizes.empty()) sizes.push_back(1);
    else sizes[0] = 4;
  } else if (count % 3 == 2) {
    sizes.push_back(2);
  }
  int32_t s = step;
  for (uint32_t k : sizes) {
    std::vector<uint64_t> st;
    for (int32_t m = 1; m < (1 << k); ++m) st.push_back(h_galois_elt(log_n, s * m));
    out->push_back(st);
    s *= 1 << k;
  }
}

static int lr_gal(he_ctx* c, const LrPlan& P, LrGal* gl) {
  gl->in.clear();
  gl->up.clear();
  gl->down.clear();
  rotsum_stages(c->log_n, (int32_t)P.g, P.logF, &gl->in);
  rotsum_stages(c->log_n, 1, P.logg, &gl->up);
  rotsum_stages(c->log_n, -1, P.logg, &gl->down);
  for (auto* v : {&gl->in, &gl->up, &gl->down})
    for (const auto& st : *v)
      for (uint64_t e : st)
        if (e == 1 || !galois_key(c, e)) return fail(HE_ENOKEY, "missing Galois key for the step's rotations");
  return HE_OK;
}

struct LrBufs {
  CtBatch U, T, A, Cc, B, Q, Tmp, Zcopy, Wrep;
};

static CtBatch carve(Arena& a, size_t count, uint32_t cap, uint32_t n) {
  uint64_t* p = a.take<uint64_t>(count * 2 * cap * n);
  return CtBatch{p, (uint64_t)2 * cap * n, cap, 0};
}

// The per-ciphertext part of the step for m data ciphertexts Zc with weights
// Wc (stride 0: one W for all): S_k = p(M_k) in b.Cc.
static int lr_chunk(he_ctx* c, const LrPlan& P, const LrGal& gl, CtBatch Zc, CtBatch Wc, uint32_t m, LrBufs& b,
                    Arena& ops, bool infer) {
  const uint32_t l0 = P.l0;
  auto fresh = [&]() -> Arena& {
    ops.off = 0;
    return ops;
  };
  // U = Z_k * W, then the rotate-and-sum over the F feature positions
  HE_TRY(mul_relin_batch(c, Zc, Wc, l0, m, b.U, true, fresh()));
  for (const auto& st : gl.in) {  // U <- U + its rotations, alternating buffers
    HE_TRY(rotsum_batch(c, b.U, l0 - 1, m, st.data(), (uint32_t)st.size(), b.Tmp, fresh()));
    std::swap(b.U, b.Tmp);
  }
  // T = M^2; A = c3 M; C = T A
  HE_TRY(mul_relin_batch(c, b.U, b.U, l0 - 1, m, b.T, true, fresh()));
  HE_TRY(mul_int_batch(c, b.U, b.Tmp, P.kA, l0 - 1, m));
  HE_TRY(rescale_batch(c, b.Tmp, l0 - 1, m, b.A, fresh()));
  HE_TRY(mul_relin_batch(c, b.T, b.A, l0 - 2, m, b.Cc, true, fresh()));
  // B = c1 M (dropped to l0-3); Q = c2 M^2
  HE_TRY(mul_int_batch(c, b.U, b.Tmp, P.kB, l0 - 1, m));
  HE_TRY(rescale_batch(c, b.Tmp, l0 - 1, m, b.B, fresh()));
  HE_TRY(addsub_batch(c, b.Cc, b.B, b.Cc, 0, l0 - 3, m));
  if (P.has_c2) {
    HE_TRY(mul_int_batch(c, b.T, b.Tmp, P.kQ, l0 - 2, m));
    HE_TRY(rescale_batch(c, b.Tmp, l0 - 2, m, b.Q, fresh()));
    HE_TRY(addsub_batch(c, b.Cc, b.Q, b.Cc, 0, l0 - 3, m));
  }
  HE_TRY(add_int_batch(c, b.Cc, b.Cc, P.k0, l0 - 3, m));
  (void)infer;  // S_k = p(M_k) is in b.Cc
  return HE_OK;
}

// The per-feature sum over the g samples, the mask and the replication, for
// `count` accumulated gradients G (uniform); result R (uniform, level l0-5).
static int lr_finish(he_ctx* c, const LrPlan& P, const LrGal& gl, const int64_t* mask, CtBatch G, uint32_t count,
                     CtBatch H1, CtBatch R, Arena& ops) {
  const uint32_t l0 = P.l0;
  auto fresh = [&]() -> Arena& {
    ops.off = 0;
    return ops;
  };
  for (const auto& st : gl.up) {  // G <- G + its rotations, alternating buffers
    HE_TRY(rotsum_batch(c, G, l0 - 4, count, st.data(), (uint32_t)st.size(), H1, fresh()));
    std::swap(G, H1);
  }
  HE_TRY(mul_plain_dev(c, G, mask, H1, l0 - 4, count, fresh()));
  HE_TRY(rescale_batch(c, H1, l0 - 4, count, R, fresh()));
  const CtBatch R_out = R;
  for (const auto& st : gl.down) {
    HE_TRY(rotsum_batch(c, R, l0 - 5, count, st.data(), (uint32_t)st.size(), H1, fresh()));
    std::swap(R, H1);
  }
  if (R.base != R_out.base) HE_TRY(copy_batch(c, R, R_out, l0 - 5, count));
  return HE_OK;
}

// One worker's inputs after validation.
struct Shard {
  const he_ct* Z;
  size_t nZ;
  he_ct W;       // weights at the level the step runs at (refreshed if needed)
  he_ct* W_out;
  he_ct* S_out;  // inference outputs
  uint32_t l0;
  uint32_t cid;  // refresh encryption id
  bool refresh;
  const he_ct* W_in;
};

static int check_aligned(const void* p) { return ((uintptr_t)p & 15) == 0 ? HE_OK : HE_EINVAL; }

// Runs the step for every shard.  Shards sharing (level, scales) are batched:
// their data ciphertexts go through the same kernels in chunks, each chunk's
// per-ciphertext results are summed into their shard's gradient, and the
// final stage runs once over all shards of the group.
static int lr_run(he_ctx* c, std::vector<Shard>& sh, const he_lr_config* cfg, uint32_t refresh_level,
                  Arena& pool, bool infer) {
  const uint32_t n = c->n;
  // in-process refresh of weights below the circuit's depth (Algorithm 1)
  for (size_t k = 0; k < sh.size(); ++k) {
    if (!sh[k].refresh) continue;
    const size_t words = (size_t)sh[k].W_in->level * n + 2 * n + 2 * n * 2 + n + 4 * (size_t)refresh_level * n;
    Arena a = pool;  // scratch after the refreshed buffers, reused per shard
    uint64_t* m = a.take<uint64_t>((size_t)sh[k].W_in->level * n);
    double* d = a.take<double>(n);
    double* re = a.take<double>(n);
    double2* fft = a.take<double2>(2 * n);
    int64_t* coeffs = a.take<int64_t>(n);
    int* ovf = a.take<int>(1);
    uint64_t* scratch = a.take<uint64_t>((size_t)4 * refresh_level * n);
    (void)words;
    if (!scratch) return fail(HE_ENOMEM, "refresh scratch too small");
    HE_TRY(decrypt_dev(c, sh[k].W_in, m, d));
    HE_TRY(decode_dev(c, d, sh[k].W_in->scale, re, n / 2, fft));
    HE_TRY(encode_dev(c, re, n / 2, sh[k].W.scale, coeffs, fft, ovf));
    HE_TRY(encrypt_dev(c, coeffs, refresh_level, 0, sh[k].cid, &sh[k].W, scratch));
  }
  // groups of shards that share the plan
  std::vector<bool> done(sh.size(), false);
  for (size_t k0 = 0; k0 < sh.size(); ++k0) {
    if (done[k0]) continue;
    std::vector<size_t> grp;
    for (size_t k = k0; k < sh.size(); ++k)
      if (!done[k] && sh[k].l0 == sh[k0].l0 && sh[k].Z[0].scale == sh[k0].Z[0].scale &&
          sh[k].W.scale == sh[k0].W.scale) {
        grp.push_back(k);
        done[k] = true;
      }
    const uint32_t l0 = sh[k0].l0;
    LrPlan P;
    HE_TRY(lr_plan(c, l0, sh[k0].Z[0].scale, sh[k0].W.scale, cfg, infer, &P));
    LrGal gl;
    HE_TRY(lr_gal(c, P, &gl));
    const int64_t* mask = nullptr;
    HE_TRY(lr_mask(c, P.g, cfg->mask_scale, &mask));
    size_t total = 0;
    for (size_t k : grp) total += sh[k].nZ;
    const uint32_t ns = (uint32_t)grp.size();
    Arena a = pool;
    CtBatch G = carve(a, ns, l0 - 4, n), H1 = carve(a, ns, l0 - 4, n), R = carve(a, ns, l0 - 4, n);
    // three-part sums D = sum_k tensor(S_k, Z_k) per shard, relinearised once
    const uint64_t d3_stride = (uint64_t)3 * (l0 - 3) * n;
    uint64_t* D3 = a.take<uint64_t>((size_t)ns * d3_stride);
    const size_t per = (lr_ct_words(c, l0) + lr_op_words(c, l0, 1, 1)) * sizeof(uint64_t);
    size_t chunk = std::max<size_t>(1, std::min(c->lr_chunk ? (size_t)c->lr_chunk : c->chunk_bytes / per, total));
    LrBufs b;
    b.U = carve(a, chunk, l0 - 1, n);
    b.T = carve(a, chunk, l0 - 2, n);
    b.A = carve(a, chunk, l0 - 2, n);
    b.Cc = carve(a, chunk, l0 - 3, n);
    b.B = carve(a, chunk, l0 - 2, n);
    b.Q = carve(a, chunk, l0 - 3, n);
    b.Tmp = carve(a, chunk, l0 - 1, n);
    b.Zcopy = carve(a, chunk, l0, n);
    b.Wrep = carve(a, chunk, l0, n);
    Arena ops;
    ops.base = a.base + a.off;
    ops.size = a.size > a.off ? a.size - a.off : 0;
    if (!b.Wrep.base || ops.size < lr_op_words(c, l0, (uint32_t)chunk, ns) * sizeof(uint64_t))
      return fail(HE_ENOMEM, "step scratch too small");
    if (!D3) return fail(HE_ENOMEM, "step scratch too small");
    HE_CUDA(cudaMemsetAsync(D3, 0, sizeof(uint64_t) * d3_stride * ns, c->stream));
    // walk the group's data ciphertexts chunk by chunk (a pipelined host
    // input may ask for a shorter first chunk: only its copy is not overlapped)
    size_t gi = 0, idx = 0;  // shard position in grp, ciphertext index in that shard
    size_t lim = c->io_first_chunk ? std::min(c->io_first_chunk, chunk) : chunk;
    bool time_first = c->io_first_chunk && c->io_time[2];  // the first chunk's arithmetic, timed
    while (gi < grp.size()) {
      // segments of this chunk: (group position, first ciphertext, count)
      std::vector<std::pair<size_t, std::pair<size_t, size_t>>> seg;
      size_t m = 0;
      while (m < lim && gi < grp.size()) {
        const Shard& s = sh[grp[gi]];
        const size_t take = std::min(lim - m, s.nZ - idx);
        seg.push_back({gi, {idx, take}});
        m += take;
        idx += take;
        if (idx == s.nZ) {
          ++gi;
          idx = 0;
        }
      }
      CtBatch Zc, Wc;
      CtBatch zu;
      const Shard& s0 = sh[grp[seg[0].first]];
      if (seg.size() == 1 && uniform_view(s0.Z + seg[0].second.first, seg[0].second.second, &zu)) {
        Zc = zu;
        Wc = CtBatch{s0.W.data, 0, s0.W.cap, 0};
      } else {
        size_t off = 0;
        for (auto& sg : seg) {
          const Shard& s = sh[grp[sg.first]];
          const size_t first = sg.second.first, cnt = sg.second.second;
          CtBatch dz = b.Zcopy, dw = b.Wrep;
          dz.base += off * b.Zcopy.stride;
          dw.base += off * b.Wrep.stride;
          if (uniform_view(s.Z + first, cnt, &zu)) {
            HE_TRY(copy_batch(c, zu, dz, l0, (uint32_t)cnt));
          } else {
            for (size_t i = 0; i < cnt; ++i) {
              CtBatch one{s.Z[first + i].data, 0, s.Z[first + i].cap, 0}, d1 = dz;
              d1.base += i * b.Zcopy.stride;
              HE_TRY(copy_batch(c, one, d1, l0, 1));
            }
          }
          HE_TRY(copy_batch(c, CtBatch{s.W.data, 0, s.W.cap, 0}, dw, l0, (uint32_t)cnt));
          off += cnt;
        }
        Zc = b.Zcopy;
        Wc = b.Wrep;
      }
      if (c->io_piece) {  // pipelined host input (one shard): wait for the pieces this chunk reads
        const size_t last = seg.back().second.first + seg.back().second.second;  // ciphertexts [0, last) needed
        const size_t need = (last + c->io_piece - 1) / c->io_piece;
        if (need > c->io_pieces_waited) {
          HE_CUDA(cudaStreamWaitEvent(c->stream, c->io_events[need - 1], 0));
          c->io_pieces_waited = need;
        }
      }
      if (time_first) HE_CUDA(cudaEventRecord(c->io_time[2], c->stream));
      HE_TRY(lr_chunk(c, P, gl, Zc, Wc, (uint32_t)m, b, ops, infer));
      if (time_first) {
        HE_CUDA(cudaEventRecord(c->io_time[3], c->stream));
        c->io_timed_first = m;
        time_first = false;
      }
      lim = chunk;
      size_t off = 0;
      if (infer) {  // copy S_k of each segment's ciphertexts to their outputs
        for (auto& sg : seg) {
          const Shard& s = sh[grp[sg.first]];
          for (size_t i = 0; i < sg.second.second; ++i) {
            CtBatch src = b.Cc;
            src.base += (off + i) * b.Cc.stride;
            he_ct& o = s.S_out[sg.second.first + i];
            HE_TRY(copy_batch(c, src, CtBatch{o.data, 0, o.cap, 0}, l0 - 3, 1));
          }
          off += sg.second.second;
        }
        continue;
      }
      for (auto& sg : seg) {  // D += tensor(S_k, Z_k) of each segment's ciphertexts
        CtBatch sk = b.Cc, zk = Zc;
        sk.base += off * b.Cc.stride;
        zk.base += off * Zc.stride;
        HE_TRY(tensor_acc_batch(c, sk, zk, (uint32_t)sg.second.second, D3 + sg.first * d3_stride, l0 - 3));
        off += sg.second.second;
      }
    }
    if (infer) continue;
    {  // G = rescale(relinearise(D))
      Arena ar = ops;
      ar.off = 0;
      HE_TRY(relin_rescale_batch(c, D3, d3_stride, l0 - 3, ns, G, ar));
    }
    HE_TRY(lr_finish(c, P, gl, mask, G, ns, H1, R, ops));
    for (uint32_t i = 0; i < ns; ++i) {
      Shard& s = sh[grp[i]];
      CtBatch r = R;
      r.base += (size_t)i * R.stride;
      HE_TRY(addsub_batch(c, CtBatch{s.W.data, 0, s.W.cap, 0}, r, CtBatch{s.W_out->data, 0, s.W_out->cap, 0}, 0,
                          l0 - 5, 1));
      if (P.kR) {  // the regulariser's gradient (Eq. 6, 8): W_out += rescale(drop(W, l0-4) * kR)
        ops.off = 0;
        uint64_t* wt = ops.take<uint64_t>((size_t)2 * (l0 - 4) * c->n);
        uint64_t* wr = ops.take<uint64_t>((size_t)2 * (l0 - 5) * c->n);
        if (!wt || !wr) return fail(HE_ENOMEM, "regulariser scratch too small");
        const CtBatch Wt{wt, 0, l0 - 4, 0}, Wr{wr, 0, l0 - 5, 0}, Wo{s.W_out->data, 0, s.W_out->cap, 0};
        HE_TRY(mul_int_batch(c, CtBatch{s.W.data, 0, s.W.cap, 0}, Wt, P.kR, l0 - 4, 1));
        HE_TRY(rescale_batch(c, Wt, l0 - 4, 1, Wr, ops));
        HE_TRY(addsub_batch(c, Wo, Wr, Wo, 0, l0 - 5, 1));
      }
    }
  }
  return HE_OK;
}

// Workspace words lr_run needs for these shards.
static size_t lr_words(he_ctx* c, const LrShape* sh, size_t count, uint32_t refresh_level) {
  const size_t n = c->n;
  size_t need = 0;
  std::map<uint32_t, std::pair<size_t, size_t>> groups;  // l0 -> (shards, ciphertexts)
  for (size_t k = 0; k < count; ++k) {
    groups[sh[k].l0].first += 1;
    groups[sh[k].l0].second += sh[k].nZ;
  }
  for (auto& kv : groups) {
    const uint32_t l0 = kv.first;
    const size_t per = (lr_ct_words(c, l0) + lr_op_words(c, l0, 1, 1)) * sizeof(uint64_t);
    const size_t chunk = std::max<size_t>(
        1, std::min(c->lr_chunk ? (size_t)c->lr_chunk : c->chunk_bytes / per, kv.second.second));
    const size_t w = 3 * kv.second.first * 2 * (l0 - 4) * n + kv.second.first * 3 * (l0 - 3) * n + 32 +
                     chunk * lr_ct_words(c, l0) +
                     lr_op_words(c, l0, (uint32_t)chunk, (uint32_t)kv.second.first) + 4096;
    need = std::max(need, w);
  }
  const size_t ref = (size_t)c->L * n + 2 * n + 4 * n + n + 4 * (size_t)refresh_level * n + 4096;
  return std::max(need, ref);
}

size_t lr_ws_bytes(he_ctx* c, const LrShape* sh, size_t count, uint32_t refresh_level) {
  size_t nref = 0;
  for (size_t k = 0; k < count; ++k) nref += sh[k].refresh;
  const size_t ref_words = nref * 2 * (size_t)refresh_level * c->n;
  return (lr_words(c, sh, count, refresh_level) + ref_words + 8192) * sizeof(uint64_t);
}

static int validate_shard(he_ctx* c, const he_lr_shard& in, const he_lr_config* cfg, uint32_t refresh_level,
                          bool infer, Shard* out) {
  if (!in.Z || in.nZ == 0 || !in.W || !in.W->data) return fail(HE_EINVAL, "shard: null argument or no data ciphertexts");
  if (!infer && (!in.W_out || !in.W_out->data)) return fail(HE_EINVAL, "shard: null output");
  if (infer) {
    if (!in.S_out) return fail(HE_EINVAL, "shard: null inference outputs");
    for (size_t k = 0; k < in.nZ; ++k)
      if (!in.S_out[k].data || ((uintptr_t)in.S_out[k].data & 15)) return fail(HE_EINVAL, "shard: bad inference output");
  }
  const uint32_t need = std::max<uint32_t>(infer ? 5 : 6, in.min_level);
  const uint32_t zl = in.Z[0].level;
  for (size_t k = 0; k < in.nZ; ++k) {
    const he_ct& z = in.Z[k];
    if (!z.data || z.level != zl || z.cap < z.level || z.level > (uint32_t)c->L)
      return fail(HE_EINVAL, "shard: data ciphertexts must share one level");
    if (check_aligned(z.data)) return fail(HE_EINVAL, "ciphertext data must be 16-byte aligned");
    if (!scales_eq(z.scale, in.Z[0].scale)) return fail(HE_ESCALE, "data ciphertexts at different scales");
  }
  if (check_aligned(in.W->data) || (!infer && check_aligned(in.W_out->data)))
    return fail(HE_EINVAL, "ciphertext data must be 16-byte aligned");
  out->Z = in.Z;
  out->nZ = in.nZ;
  out->W_in = in.W;
  out->W_out = in.W_out;
  out->S_out = in.S_out;
  out->cid = in.refresh_cid;
  out->W = *in.W;
  out->refresh = false;
  uint32_t wl = in.W->level;
  if (wl < need) {
    if (!refresh_level) return fail(HE_ELEVEL, "too few levels left: refresh the weights");
    if (refresh_level < need || refresh_level > zl) return fail(HE_EINVAL, "refresh level out of range");
    out->refresh = true;
    wl = refresh_level;
  }
  if (wl > zl) return fail(HE_EINVAL, "weights above the data's level");
  out->l0 = wl;
  if (!infer && in.W_out->cap < wl - 5) return fail(HE_EINVAL, "output capacity too small");
  if (infer)
    for (size_t k = 0; k < in.nZ; ++k)
      if (in.S_out[k].cap < wl - 3) return fail(HE_EINVAL, "inference output capacity too small");
  const uint32_t g = cfg->g;
  if (g < 1 || (g & (g - 1)) || g > (uint32_t)c->n / 2) return fail(HE_EINVAL, "g must be a power of two <= N/2");
  if (!(cfg->mask_scale > 0.0)) return fail(HE_EINVAL, "mask_scale must be positive");
  if (!(cfg->l2 >= 0.0) || !std::isfinite(cfg->l2)) return fail(HE_EINVAL, "l2 must be finite and >= 0");
  return HE_OK;
}

int lr_entry(he_ctx* c, const he_lr_shard* shards, size_t count, const he_lr_config* cfg,
             uint32_t refresh_level, int flags, bool infer) {
  if (!c || !shards || !cfg || count == 0) return fail(HE_EINVAL, "he_lr: null argument");
  std::vector<Shard> sh(count);
  for (size_t k = 0; k < count; ++k) HE_TRY(validate_shard(c, shards[k], cfg, refresh_level, infer, &sh[k]));
  // plans, keys and masks are checked (and masks encoded) before any capture
  for (size_t k = 0; k < count; ++k) {
    LrPlan P;
    HE_TRY(lr_plan(c, sh[k].l0, sh[k].Z[0].scale, sh[k].refresh ? sh[k].W_in->scale : sh[k].W.scale, cfg, infer, &P));
    LrGal gl;
    HE_TRY(lr_gal(c, P, &gl));
    const int64_t* mask = nullptr;
    HE_TRY(lr_mask(c, P.g, cfg->mask_scale, &mask));
  }
  // refreshed weights live in a context-owned buffer per shard
  std::vector<LrShape> shapes(count);
  for (size_t k = 0; k < count; ++k) shapes[k] = LrShape{sh[k].l0, sh[k].nZ, sh[k].refresh};
  HE_TRY(ws_reserve(c, lr_ws_bytes(c, shapes.data(), count, refresh_level)));
  Arena pool;
  pool.base = (char*)c->ws.ptr;
  pool.size = c->ws.size;
  for (auto& s : sh) {
    if (!s.refresh) continue;
    uint64_t* p = pool.take<uint64_t>(2 * (size_t)refresh_level * c->n);
    s.W = he_ct{p, refresh_level, refresh_level, s.W_in->scale};
  }
  Arena rest;
  rest.base = pool.base + pool.off;
  rest.size = pool.size - pool.off;
  const bool graph = (flags & HE_LR_GRAPH) && c->stream != nullptr;
  if (!graph) {
    HE_TRY(lr_run(c, sh, cfg, refresh_level, rest, infer));
  } else {
    // one CUDA graph per distinct call (pointers, sizes, configuration)
    std::string key;
    char buf[160];
    snprintf(buf, sizeof buf, "%d|%u|%a|%a|%a|%a|%a|%a|%u|%a|", (int)infer, refresh_level, cfg->coeffs[0],
             cfg->coeffs[1], cfg->coeffs[2], cfg->coeffs[3], cfg->lr, cfg->mask_scale, cfg->g, cfg->l2);
    key += buf;
    for (auto& s : sh) {
      snprintf(buf, sizeof buf, "%p,%zu,%p,%u,%a,%p,%p,%u;", (const void*)s.Z, s.nZ, (const void*)s.W_in->data,
               s.W_in->level, s.W_in->scale, (const void*)(s.W_out ? s.W_out->data : nullptr),
               (const void*)s.S_out, s.cid);
      key += buf;
      for (size_t i = 0; i < s.nZ; ++i) {
        snprintf(buf, sizeof buf, "%p/%u/%u/%a,", (const void*)s.Z[i].data, s.Z[i].level, s.Z[i].cap, s.Z[i].scale);
        key += buf;
      }
    }
    snprintf(buf, sizeof buf, "ws=%p", c->ws.ptr);
    key += buf;
    auto it = c->graphs.find(key);
    if (it == c->graphs.end()) {
      const bool prof = c->prof_on;
      c->prof_on = false;
      cudaGraph_t g = nullptr;
      HE_CUDA(cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
      const int rc = lr_run(c, sh, cfg, refresh_level, rest, infer);
      const cudaError_t ce = cudaStreamEndCapture(c->stream, &g);
      c->prof_on = prof;
      if (rc != HE_OK) {
        if (g) cudaGraphDestroy(g);
        return rc;
      }
      if (ce != cudaSuccess) return fail(HE_ECUDA, std::string("graph capture: ") + cudaGetErrorString(ce));
      cudaGraphExec_t ex = nullptr;
      const cudaError_t ie = cudaGraphInstantiate(&ex, g, 0);
      cudaGraphDestroy(g);
      if (ie != cudaSuccess) return fail(HE_ECUDA, std::string("graph instantiate: ") + cudaGetErrorString(ie));
      it = c->graphs.emplace(key, ex).first;
    }
    HE_CUDA(cudaGraphLaunch(it->second, c->stream));
  }
  for (size_t k = 0; k < count; ++k) {
    if (infer) {
      LrPlan P;
      HE_TRY(lr_plan(c, sh[k].l0, sh[k].Z[0].scale, sh[k].W.scale, cfg, true, &P));
      for (size_t i = 0; i < sh[k].nZ; ++i) {
        shards[k].S_out[i].level = sh[k].l0 - 3;
        shards[k].S_out[i].scale = P.sC;
      }
    } else {
      shards[k].W_out->level = sh[k].l0 - 5;
      shards[k].W_out->scale = sh[k].W.scale;
    }
  }
  return HE_OK;
}

}  // namespace he

using namespace he;

extern "C" int he_lr_gradient_step(he_ctx* c, const he_ct* Z, size_t nZ, const he_ct* W, const he_lr_config* cfg,
                                   he_ct* W_out) {
  if (!c || !Z || !W || !cfg || !W_out) return fail(HE_EINVAL, "he_lr_gradient_step: null argument");
  if (W->level < 6) return fail(HE_ELEVEL, "the step needs inputs at level >= 6");
  for (size_t k = 0; k < nZ; ++k)
    if (Z[k].level != W->level) return fail(HE_EINVAL, "data and weights must share one level");
  he_lr_shard s{Z, nZ, W, W_out, nullptr, 0, 0};
  return lr_entry(c, &s, 1, cfg, 0, 0, false);
}

// The step with its inputs and output in host memory: the weights, then the
// data ciphertexts in pieces, are copied on a second stream while the circuit
// runs chunk by chunk on the context's stream (a short first chunk, then
// chunks of the scratch budget), each chunk waiting only for the pieces it
// reads; the new weights are copied back at the end.
extern "C" int he_lr_gradient_step_host(he_ctx* c, const uint64_t* Z, size_t nZ, uint32_t z_level, double z_scale,
                                        const uint64_t* W, uint32_t w_level, double w_scale,
                                        const he_lr_config* cfg, uint64_t* out, size_t out_words,
                                        uint32_t* out_level, double* out_scale) {
  if (!c || !Z || !W || !cfg || !out || nZ == 0) return fail(HE_EINVAL, "he_lr_gradient_step_host: null argument");
  if (z_level < 6 || z_level > (uint32_t)c->L || w_level < 6 || w_level > z_level)
    return fail(w_level < 6 ? HE_ELEVEL : HE_EINVAL, "he_lr_gradient_step_host: bad levels");
  const size_t n = c->n, zw = (size_t)2 * z_level * n, ww = (size_t)2 * w_level * n;
  const uint32_t lo = w_level - 5;
  if (out_words < (size_t)2 * lo * n) return fail(HE_EINVAL, "he_lr_gradient_step_host: output buffer too small");
  const size_t words = zw * nZ + ww + 2 * (size_t)lo * n + 64;
  if (c->io.size < words * sizeof(uint64_t)) {
    HE_CUDA(cudaStreamSynchronize(c->stream));
    if (c->copy_stream) HE_CUDA(cudaStreamSynchronize(c->copy_stream));
    cudaFree(c->io.ptr);
    c->io.ptr = nullptr;
    c->io.size = 0;
    if (cudaMalloc(&c->io.ptr, words * sizeof(uint64_t)) != cudaSuccess) {
      cudaGetLastError();
      return fail(HE_ENOMEM, "he_lr_gradient_step_host: device input buffer");
    }
    c->io.size = words * sizeof(uint64_t);
  }
  if (!c->copy_stream) HE_CUDA(cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking));
  const size_t piece = 16;  // data ciphertexts per copy (32 MB at N = 2^14, 8 limbs)
  const size_t pieces = (nZ + piece - 1) / piece;
  while (c->io_events.size() < pieces + 1) {
    cudaEvent_t e;
    HE_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    c->io_events.push_back(e);
  }
  uint64_t* dZ = (uint64_t*)c->io.ptr;
  uint64_t* dW = dZ + zw * nZ;
  uint64_t* dO = dW + ww;
  for (cudaEvent_t& e : c->io_time)
    if (!e) HE_CUDA(cudaEventCreate(&e));
  // the first chunk (whole pieces): only its copy is exposed, the rest's copy
  // overlaps its arithmetic.  From the previous call's timings, the smallest
  // f with (nZ - f) * copy <= f * arithmetic per ciphertext; else an eighth.
  size_t first_chunk = std::max(piece, nZ / 8 / piece * piece);
  if (c->io_timed_nZ && c->io_timed_first) {
    float copy_ms = 0.f, arith_ms = 0.f;
    if (cudaEventElapsedTime(&copy_ms, c->io_time[0], c->io_time[1]) == cudaSuccess &&
        cudaEventElapsedTime(&arith_ms, c->io_time[2], c->io_time[3]) == cudaSuccess && copy_ms > 0.f &&
        arith_ms > 0.f) {
      const double cp = copy_ms / (double)c->io_timed_nZ, ar = arith_ms / (double)c->io_timed_first;
      const size_t f = (size_t)ceil((double)nZ * cp / (cp + ar) / (double)piece) * piece;
      first_chunk = std::min(std::max(f, piece), std::max(piece, nZ / 2 / piece * piece));
    } else {
      cudaGetLastError();  // events of a call that failed: keep the default
    }
  }
  c->io_timed_nZ = c->io_timed_first = 0;
  // the copy stream may overwrite the buffers only after the previous step on c->stream is done with them
  HE_CUDA(cudaEventRecord(c->io_events[pieces], c->stream));
  HE_CUDA(cudaStreamWaitEvent(c->copy_stream, c->io_events[pieces], 0));
  HE_CUDA(cudaEventRecord(c->io_time[0], c->copy_stream));
  HE_CUDA(cudaMemcpyAsync(dW, W, sizeof(uint64_t) * ww, cudaMemcpyHostToDevice, c->copy_stream));
  for (size_t k = 0; k < pieces; ++k) {
    const size_t first = k * piece, cnt = std::min(piece, nZ - first);
    HE_CUDA(cudaMemcpyAsync(dZ + first * zw, Z + first * zw, sizeof(uint64_t) * zw * cnt, cudaMemcpyHostToDevice,
                            c->copy_stream));
    HE_CUDA(cudaEventRecord(c->io_events[k], c->copy_stream));
  }
  HE_CUDA(cudaEventRecord(c->io_time[1], c->copy_stream));
  std::vector<he_ct> zc(nZ);
  for (size_t i = 0; i < nZ; ++i) zc[i] = he_ct{dZ + i * zw, z_level, z_level, z_scale};
  he_ct wc{dW, w_level, w_level, w_scale}, oc{dO, 0, lo, 0.0};
  he_lr_shard sh{zc.data(), nZ, &wc, &oc, nullptr, 0, 0};
  // the weights arrive with the first piece's copy ordering: wait for it before the step
  HE_CUDA(cudaStreamWaitEvent(c->stream, c->io_events[0], 0));
  c->io_piece = piece;
  c->io_pieces_waited = 1;
  // unless the caller chose a chunk: the short first chunk, then chunks of
  // the scratch budget
  if (!c->lr_chunk && nZ > 2 * piece) c->io_first_chunk = first_chunk;
  const int rc = lr_entry(c, &sh, 1, cfg, 0, 0, false);
  c->io_first_chunk = 0;
  c->io_piece = 0;
  if (rc == HE_OK && c->io_timed_first) c->io_timed_nZ = nZ;
  if (rc != HE_OK) {
    cudaStreamSynchronize(c->copy_stream);
    return rc;
  }
  HE_CUDA(cudaMemcpyAsync(out, dO, sizeof(uint64_t) * 2 * lo * n, cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  if (out_level) *out_level = oc.level;
  if (out_scale) *out_scale = oc.scale;
  return HE_OK;
}

extern "C" int he_lr_gradient_step_workers(he_ctx* c, const he_lr_shard* shards, size_t count,
                                           const he_lr_config* cfg, uint32_t refresh_level, int flags) {
  return lr_entry(c, shards, count, cfg, refresh_level, flags, false);
}

extern "C" int he_lr_inference_workers(he_ctx* c, const he_lr_shard* shards, size_t count, const he_lr_config* cfg,
                                       uint32_t refresh_level, int flags) {
  return lr_entry(c, shards, count, cfg, refresh_level, flags, true);
}

// ---- the training loop of Algorithms 1 and 2 ---------------------------------

namespace he {

__global__ void k_slots_accumulate(double* acc, const double* x, size_t n, int first, double scale_after) {
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < n; g += (size_t)gridDim.x * blockDim.x) {
    const double v = first ? x[g] : acc[g] + x[g];
    acc[g] = scale_after != 0.0 ? v * scale_after : v;
  }
}

// The key holder's round (Algorithm 2): decrypt every worker's
// weights, average them slot by slot (in worker order), encode the average at
// `scale` and encrypt it once at `level` (stream cid) into W[0], then copy it
// to every other worker.
static int lr_aggregate(he_ctx* c, std::vector<he_ct>& W, uint32_t level, double scale, uint32_t cid) {
  const size_t n = c->n, ns = n / 2;
  size_t lmax = 0;
  for (const he_ct& w : W) lmax = std::max<size_t>(lmax, w.level);
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * lmax * n + sizeof(double) * (n + 2 * ns) + sizeof(double2) * 2 * n +
                           sizeof(int64_t) * n + sizeof(uint64_t) * 4 * level * n + 16384));
  Arena ar;
  ar.base = (char*)c->ws.ptr;
  ar.size = c->ws.size;
  ar.off = 0;
  uint64_t* m = ar.take<uint64_t>(lmax * n);
  double* d = ar.take<double>(n);
  double* re = ar.take<double>(ns);
  double* avg = ar.take<double>(ns);
  double2* fft = ar.take<double2>(2 * n);
  int64_t* coeffs = ar.take<int64_t>(n);
  int* ovf = ar.take<int>(1);
  uint64_t* scratch = ar.take<uint64_t>((size_t)4 * level * n);
  if (!scratch) return fail(HE_ENOMEM, "aggregation scratch too small");
  for (size_t k = 0; k < W.size(); ++k) {
    HE_TRY(decrypt_dev(c, &W[k], m, d));
    HE_TRY(decode_dev(c, d, W[k].scale, re, ns, fft));
    const bool last = k + 1 == W.size();
    k_slots_accumulate<<<grid_for(ns), 256, 0, c->stream>>>(avg, re, ns, k == 0, last ? 1.0 / (double)W.size() : 0.0);
    HE_CUDA(cudaGetLastError());
  }
  HE_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c->stream));
  HE_TRY(encode_dev(c, avg, ns, scale, coeffs, fft, ovf));
  HE_TRY(encrypt_dev(c, coeffs, level, 0, cid, &W[0], scratch));
  W[0].level = level;
  W[0].scale = scale;
  for (size_t k = 1; k < W.size(); ++k) {
    HE_TRY(copy_batch(c, CtBatch{W[0].data, 0, W[0].cap, 0}, CtBatch{W[k].data, 0, W[k].cap, 0}, level, 1));
    W[k].level = level;
    W[k].scale = scale;
  }
  HE_TRY(stage_reserve(c, 64));
  HE_CUDA(cudaMemcpyAsync(c->h_stage, ovf, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  int flag = 0;
  memcpy(&flag, c->h_stage, sizeof(int));
  return flag ? fail(HE_EINVAL, "aggregation: encoded coefficient beyond int64") : HE_OK;
}

}  // namespace he

// Algorithms 1 and 2 in one process: every worker k runs `iterations`
// gradient steps (Eq. 7-8) on its own data Z_k from its own weights; after
// every `refresh_every` steps, and after the last, the key holder replaces
// all workers' weights by the re-encrypted slot-wise average of their
// weights (the paper leaves the parameter server's update rule open).
extern "C" int he_lr_train(he_ctx* c, const he_lr_shard* shards, size_t count, const he_lr_config* cfg,
                           uint32_t iterations, uint32_t refresh_every, uint32_t top_level, uint32_t cid0,
                           he_ct* W_final) {
  if (!c || !shards || !cfg || !W_final || count == 0 || iterations == 0 || refresh_every == 0)
    return fail(HE_EINVAL, "he_lr_train: null argument or zero count");
  if (top_level < 6 || top_level > (uint32_t)c->L) return fail(HE_EINVAL, "he_lr_train: top level out of range");
  if (top_level < 5 * refresh_every + 1)
    return fail(HE_ELEVEL, "he_lr_train: the weights run out of limbs before the refresh");
  if (!W_final->data || W_final->cap < top_level) return fail(HE_EINVAL, "he_lr_train: output capacity too small");
  const size_t n = c->n, words = (size_t)2 * top_level * n;
  double scale = 0.0;
  for (size_t k = 0; k < count; ++k) {
    const he_ct* w = shards[k].W;
    if (!w || !w->data || w->level != top_level) return fail(HE_EINVAL, "he_lr_train: weights must be at the top level");
    if (k == 0) scale = w->scale;
    else if (w->scale != scale) return fail(HE_ESCALE, "he_lr_train: workers' weights at different scales");
  }
  uint64_t* buf = nullptr;
  if (cudaMalloc(&buf, sizeof(uint64_t) * words * 2 * count) != cudaSuccess) {
    cudaGetLastError();
    return fail(HE_ENOMEM, "he_lr_train: weight buffers");
  }
  std::vector<he_ct> cur(count), nxt(count);
  int rc = HE_OK;
  for (size_t k = 0; k < count && rc == HE_OK; ++k) {
    cur[k] = he_ct{buf + 2 * k * words, top_level, top_level, scale};
    nxt[k] = he_ct{buf + (2 * k + 1) * words, 0, top_level, 0.0};
    rc = copy_batch(c, CtBatch{shards[k].W->data, 0, shards[k].W->cap, 0}, CtBatch{cur[k].data, 0, top_level, 0},
                    top_level, 1);
  }
  std::vector<he_lr_shard> sh(count);
  for (uint32_t it = 1; it <= iterations && rc == HE_OK; ++it) {
    for (size_t k = 0; k < count; ++k) sh[k] = he_lr_shard{shards[k].Z, shards[k].nZ, &cur[k], &nxt[k], nullptr, 0, 0};
    rc = lr_entry(c, sh.data(), count, cfg, 0, 0, false);
    if (rc != HE_OK) break;
    std::swap(cur, nxt);
    if (it % refresh_every == 0 || it == iterations) rc = lr_aggregate(c, cur, top_level, scale, cid0 + it);
  }
  if (rc == HE_OK)
    rc = copy_batch(c, CtBatch{cur[0].data, 0, top_level, 0}, CtBatch{W_final->data, 0, W_final->cap, 0}, top_level, 1);
  if (rc == HE_OK) {
    W_final->level = top_level;
    W_final->scale = scale;
  }
  cudaStreamSynchronize(c->stream);
  cudaFree(buf);
  return rc;
}
