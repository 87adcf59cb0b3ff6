// api.cu -- the extern "C" entry points declared in include/he_gb300.h.
// Argument checking, workspace carving and host<->device staging; every
// residue operation is delegated to the kernels through ops.cu.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "he_ops.h"

namespace he {

static thread_local std::string g_err;

void set_error(const std::string& msg) { g_err = msg; }

int fail(int code, const std::string& msg) {
  g_err = msg;
  return code;
}

size_t ws_alloc_bytes(size_t bytes) { return bytes + bytes / 8 + (1 << 20); }

int ws_reserve(he_ctx* c, size_t bytes) {
  c->ws_requests += 1;
  if (c->ws.size >= bytes) return HE_OK;
  HE_CUDA(cudaStreamSynchronize(c->stream));
  if (c->ws.ptr) cudaFree(c->ws.ptr);
  c->ws.ptr = nullptr;
  c->ws.size = 0;
  const size_t want = ws_alloc_bytes(bytes);
  if (cudaMalloc(&c->ws.ptr, want) != cudaSuccess) {
    cudaGetLastError();
    c->ws.ptr = nullptr;
    return fail(HE_ENOMEM, "workspace allocation failed");
  }
  c->ws.size = want;
  return HE_OK;
}

int stage_reserve(he_ctx* c, size_t bytes) {
  if (c->h_stage_size >= bytes) return HE_OK;
  HE_CUDA(cudaStreamSynchronize(c->stream));
  if (c->h_stage) cudaFreeHost(c->h_stage);
  c->h_stage = nullptr;
  c->h_stage_size = 0;
  HE_CUDA(cudaMallocHost(&c->h_stage, bytes));
  c->h_stage_size = bytes;
  return HE_OK;
}

static Arena arena(he_ctx* c) {
  Arena a;
  a.base = (char*)c->ws.ptr;
  a.size = c->ws.size;
  a.off = 0;
  return a;
}

static bool aligned16(const void* p) { return ((uintptr_t)p & 15) == 0; }

static int check_ct(const he_ctx* c, const he_ct* a, const char* what) {
  if (!a || !a->data) return fail(HE_EINVAL, std::string(what) + ": null ciphertext");
  if (!aligned16(a->data)) return fail(HE_EINVAL, std::string(what) + ": data must be 16-byte aligned");
  if (a->level < 1 || a->level > (uint32_t)c->L || a->cap < a->level)
    return fail(HE_EINVAL, std::string(what) + ": bad level or capacity");
  return HE_OK;
}

static int check_out(const he_ctx* c, he_ct* o, uint32_t level, const char* what) {
  if (!o || !o->data) return fail(HE_EINVAL, std::string(what) + ": null output");
  if (!aligned16(o->data)) return fail(HE_EINVAL, std::string(what) + ": output must be 16-byte aligned");
  if (o->cap < level || level < 1 || level > (uint32_t)c->L)
    return fail(HE_EINVAL, std::string(what) + ": output capacity too small");
  return HE_OK;
}

static bool scales_match(double a, double b) { return fabs(a / b - 1.0) < ldexp(1.0, -40); }

static CtBatch one(const he_ct* a) { return CtBatch{a->data, 0, a->cap, 0}; }

// If the count ciphertexts sit at a constant stride with one capacity, return
// that uniform view.
bool uniform_view(const he_ct* a, size_t count, CtBatch* out) {
  if (count == 0) return false;
  const uint64_t* b = a[0].data;
  const int64_t stride = count > 1 ? (int64_t)(a[1].data - b) : 0;
  for (size_t i = 1; i < count; ++i)
    if (a[i].cap != a[0].cap || (int64_t)(a[i].data - b) != (int64_t)i * stride) return false;
  if (stride < 0) return false;
  *out = CtBatch{a[0].data, (uint64_t)stride, a[0].cap, 0};
  return true;
}

he_ctx* ctx_view(he_ctx* base, cudaStream_t stream) {
  he_ctx* v = new he_ctx();
  v->prm = base->prm;
  v->view = true;
  v->log_n = base->log_n;
  v->n = base->n;
  v->L = base->L;
  v->alpha = base->alpha;
  v->np = base->np;
  v->beta = base->beta;
  v->q = base->q;
  v->psi = base->psi;
  v->stream = stream;
  v->device = base->device;
  v->smem_per_sm = base->smem_per_sm;
  v->d_primes = base->d_primes;
  v->d_tw = base->d_tw;
  v->d_itw = base->d_itw;
  v->d_two64 = base->d_two64;
  v->d_gauss = base->d_gauss;
  v->gK = base->gK;
  v->modup = base->modup;
  v->d_modup = base->d_modup;
  v->d_moddown = base->d_moddown;
  v->d_rescale = base->d_rescale;
  v->d_rescale_md = base->d_rescale_md;
  v->rescale_md_words = base->rescale_md_words;
  v->d_mdrs = base->d_mdrs;
  v->mdrs_words = base->mdrs_words;
  v->d_garner = base->d_garner;
  v->chunk_bytes = base->chunk_bytes;
  v->lr_chunk = base->lr_chunk;
  v->ntt_generic = base->ntt_generic;
  v->ntt_shape = base->ntt_shape;
  v->ntt_pb_max = base->ntt_pb_max;
  v->ks_ct = base->ks_ct;
  v->P_mod_q = base->P_mod_q;
  v->d_s = base->d_s;
  v->d_pk = base->d_pk;
  v->d_rlk = base->d_rlk;
  v->gal = base->gal;
  return v;
}

static void destroy(he_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  if (c->copy_stream) cudaStreamSynchronize(c->copy_stream);
  for (cudaEvent_t e : c->io_events) cudaEventDestroy(e);
  for (cudaEvent_t e : c->io_time)
    if (e) cudaEventDestroy(e);
  if (c->copy_stream) cudaStreamDestroy(c->copy_stream);
  cudaFree(c->io.ptr);
  if (c->view) {  // only the view's own state
    for (auto& kv : c->lr_masks) cudaFree(kv.second);
    for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
    cudaFree(c->ws.ptr);
    if (c->h_stage) cudaFreeHost(c->h_stage);
    prof_clear(c);
    delete c;
    return;
  }
  cudaFree(c->d_primes);
  cudaFree(c->d_tw);
  cudaFree(c->d_itw);
  cudaFree(c->d_two64);
  cudaFree(c->d_gauss);
  cudaFree(c->d_modup);
  cudaFree(c->d_moddown);
  cudaFree(c->d_rescale);
  cudaFree(c->d_rescale_md);
  cudaFree(c->d_mdrs);
  cudaFree(c->d_garner);
  cudaFree(c->d_s);
  cudaFree(c->d_pk);
  cudaFree(c->d_rlk);
  for (auto& kv : c->gal) cudaFree(kv.second);
  for (auto& kv : c->lr_masks) cudaFree(kv.second);
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  cudaFree(c->ws.ptr);
  if (c->h_stage) cudaFreeHost(c->h_stage);
  prof_clear(c);
  delete c;
}

// Multiply count ciphertexts by the plaintext with device coefficients d_coeffs.
int mul_plain_dev(he_ctx* c, CtBatch A, const int64_t* d_coeffs, CtBatch O, uint32_t level, uint32_t count,
                  Arena& ar) {
  const size_t n = c->n;
  uint64_t* pt = ar.take<uint64_t>((size_t)level * n);
  if (!pt) return fail(HE_ENOMEM, "plaintext scratch too small");
  {
    ProfScope prof(c, "elementwise", 0.0, (double)level * n * 16);
    k_signed_to_residues<<<grid_for((size_t)level * n), 256, 0, c->stream>>>(d_coeffs, pt, level, c->log_n,
                                                                             c->d_primes);
    HE_CUDA(cudaGetLastError());
  }
  PolyBatch b;
  b.src = pt;
  b.dst = pt;
  b.src_stride = b.dst_stride = 0;
  b.npolys = 1;
  b.nl = level;
  b.limb0 = 0;
  b.level = c->L;
  b.skip_alpha = 0;
  b.skip_beta = 1;
  HE_TRY(ntt_forward(c, b));
  ProfScope prof(c, "elementwise", 0.0, (double)(4 * count + 1) * level * n * 8);
  k_mul_plain<<<grid_for((size_t)count * level * n), 256, 0, c->stream>>>(A, pt, O, level, count, c->log_n,
                                                                          c->d_primes);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

void ctx_destroy(he_ctx* c) { destroy(c); }

}  // namespace he

using namespace he;

extern "C" {

const char* he_last_error(void) { return g_err.c_str(); }

int he_ctx_create(const he_params* p, const int32_t* rot_steps, size_t n_rot, void* stream, he_ctx** out) {
  if (!p || !out) return fail(HE_EINVAL, "he_ctx_create: null argument");
  *out = nullptr;
  if (p->log_n < 4 || p->log_n > 16) return fail(HE_EINVAL, "log_n must be in [4, 16]");
  if (p->n_limbs < 1 || p->n_special < 1 || p->n_special > HE_MAX_DIGIT - 1 ||
      p->n_limbs + p->n_special > HE_MAX_PRIMES)
    return fail(HE_EINVAL, "bad limb / special prime counts");
  if (p->limb_bits < 20 || p->limb_bits > 61 || p->special_bits < 20 || p->special_bits > 61)
    return fail(HE_EINVAL, "prime sizes must be in [20, 61] bits");
  const uint32_t beta = (p->n_limbs + p->n_special - 1) / p->n_special;
  if (p->dnum && p->dnum != beta) return fail(HE_EINVAL, "dnum must equal ceil(L / alpha)");
  if (!(p->scale > 0.0) || !(p->sigma > 0.0)) return fail(HE_EINVAL, "scale and sigma must be positive");
  if (n_rot && !rot_steps) return fail(HE_EINVAL, "null rotation list");
  he_ctx* c = new he_ctx();
  c->prm = *p;
  c->log_n = (int)p->log_n;
  c->n = 1 << p->log_n;
  c->L = (int)p->n_limbs;
  c->alpha = (int)p->n_special;
  c->np = c->L + c->alpha;
  c->beta = (int)beta;
  c->stream = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  {
    int smem = 0;
    if (cudaDeviceGetAttribute(&smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor, c->device) == cudaSuccess && smem > 0)
      c->smem_per_sm = (size_t)smem;
  }
  int rc = build_tables(c);
  if (rc == HE_OK) {
    std::vector<int32_t> rots(rot_steps, rot_steps + n_rot);
    rc = keygen(c, rots);
  }
  if (rc != HE_OK) {
    const std::string msg = g_err;
    destroy(c);
    g_err = msg;
    return rc;
  }
  *out = c;
  return HE_OK;
}

int he_ctx_destroy(he_ctx* c) {
  destroy(c);
  return HE_OK;
}

int he_set_stream(he_ctx* c, void* stream) {
  if (!c) return fail(HE_EINVAL, "null context");
  c->stream = (cudaStream_t)stream;
  return HE_OK;
}

int he_sync(he_ctx* c) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_CUDA(cudaStreamSynchronize(c->stream));
  return HE_OK;
}

int he_set_tuning(he_ctx* c, const char* key, double value) {
  if (!c || !key) return fail(HE_EINVAL, "he_set_tuning: null argument");
  const std::string k(key);
  if (k == "chunk_bytes") {
    if (!(value >= (1 << 20) && value <= 1e13)) return fail(HE_EINVAL, "chunk_bytes out of range");
    c->chunk_bytes = (size_t)value;
  } else if (k == "ntt_generic") {
    c->ntt_generic = value != 0.0;
  } else if (k == "lr_chunk") {
    if (!(value >= 0 && value <= 1 << 20)) return fail(HE_EINVAL, "lr_chunk out of range");
    c->lr_chunk = (uint32_t)value;
  } else if (k == "ntt_shape") {
    if (value != 0.0 && value != 1.0 && value != 2.0) return fail(HE_EINVAL, "ntt_shape is 0, 1 or 2");
    c->ntt_shape = (int)value;
  } else if (k == "ntt_pb_max") {
    if (!(value >= 1 && value <= 64) || value != (double)(uint32_t)value)
      return fail(HE_EINVAL, "ntt_pb_max is an integer in [1, 64]");
    c->ntt_pb_max = (uint32_t)value;
  } else if (k == "ks_ct") {
    if (value != 0.0 && value != 1.0 && value != 2.0 && value != 4.0) return fail(HE_EINVAL, "ks_ct is 0, 1, 2 or 4");
    c->ks_ct = (uint32_t)value;
  } else {
    return fail(HE_EINVAL, "unknown tuning key " + k);
  }
  return HE_OK;
}

int he_ctx_info(const he_ctx* c, uint32_t* n, uint32_t* L, uint32_t* alpha, uint32_t* beta, uint64_t* primes) {
  if (!c) return fail(HE_EINVAL, "null context");
  if (n) *n = (uint32_t)c->n;
  if (L) *L = (uint32_t)c->L;
  if (alpha) *alpha = (uint32_t)c->alpha;
  if (beta) *beta = (uint32_t)c->beta;
  if (primes) memcpy(primes, c->q.data(), sizeof(uint64_t) * c->np);
  return HE_OK;
}

int he_ctx_workspace(const he_ctx* c, size_t* bytes, uint64_t* requests) {
  if (!c) return fail(HE_EINVAL, "he_ctx_workspace: null context");
  if (bytes) *bytes = c->ws.size;
  if (requests) *requests = c->ws_requests;
  return HE_OK;
}

int he_encode(he_ctx* c, const double* slots, size_t n_slots, double scale, int64_t* coeffs_out) {
  if (!c || (!slots && n_slots) || !coeffs_out) return fail(HE_EINVAL, "he_encode: null argument");
  const size_t n = c->n;
  HE_TRY(ws_reserve(c, sizeof(double2) * 2 * n + sizeof(double) * n + sizeof(int64_t) * n + 4096));
  Arena ar = arena(c);
  double2* fft = ar.take<double2>(2 * n);
  double* z = ar.take<double>(n);
  int64_t* m = ar.take<int64_t>(n);
  int* ovf = ar.take<int>(1);
  HE_TRY(stage_reserve(c, sizeof(int64_t) * n + 64));
  if (n_slots) {
    if (n_slots > n / 2) return fail(HE_EINVAL, "more slots than N/2");
    memcpy(c->h_stage, slots, sizeof(double) * n_slots);
    HE_CUDA(cudaMemcpyAsync(z, c->h_stage, sizeof(double) * n_slots, cudaMemcpyHostToDevice, c->stream));
  }
  HE_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c->stream));
  HE_TRY(encode_dev(c, z, n_slots, scale, m, fft, ovf));
  HE_CUDA(cudaMemcpyAsync(c->h_stage, m, sizeof(int64_t) * n, cudaMemcpyDeviceToHost, c->stream));
  int flag = 0;
  HE_CUDA(cudaMemcpyAsync((char*)c->h_stage + sizeof(int64_t) * n, ovf, sizeof(int), cudaMemcpyDeviceToHost,
                          c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(&flag, (char*)c->h_stage + sizeof(int64_t) * n, sizeof(int));
  if (flag) return fail(HE_EINVAL, "encoded coefficient beyond int64");
  memcpy(coeffs_out, c->h_stage, sizeof(int64_t) * n);
  return HE_OK;
}

int he_encrypt_poly(he_ctx* c, const int64_t* coeffs, double scale, uint32_t level, int use_sk, uint32_t cid,
                    he_ct* out) {
  if (!c || !coeffs) return fail(HE_EINVAL, "he_encrypt_poly: null argument");
  HE_TRY(check_out(c, out, level, "he_encrypt_poly"));
  const size_t n = c->n;
  HE_TRY(ws_reserve(c, sizeof(int64_t) * n + sizeof(uint64_t) * 4 * level * n + 4096));
  Arena ar = arena(c);
  int64_t* m = ar.take<int64_t>(n);
  uint64_t* scratch = ar.take<uint64_t>((size_t)4 * level * n);
  HE_TRY(stage_reserve(c, sizeof(int64_t) * n));
  memcpy(c->h_stage, coeffs, sizeof(int64_t) * n);
  HE_CUDA(cudaMemcpyAsync(m, c->h_stage, sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream));
  HE_TRY(encrypt_dev(c, m, level, use_sk, cid, out, scratch));
  out->scale = scale;
  // the staging buffer is reused by the next call: wait for the copy
  HE_CUDA(cudaStreamSynchronize(c->stream));
  return HE_OK;
}

int he_encode_encrypt(he_ctx* c, const double* slots, size_t n_slots, double scale, uint32_t level, int use_sk,
                      uint32_t cid, he_ct* out) {
  if (!c || (!slots && n_slots)) return fail(HE_EINVAL, "he_encode_encrypt: null argument");
  HE_TRY(check_out(c, out, level, "he_encode_encrypt"));
  if (n_slots > (size_t)c->n / 2) return fail(HE_EINVAL, "more slots than N/2");
  const size_t n = c->n;
  HE_TRY(ws_reserve(c, sizeof(double2) * 2 * n + sizeof(double) * n + sizeof(int64_t) * n +
                           sizeof(uint64_t) * 4 * level * n + 8192));
  Arena ar = arena(c);
  double2* fft = ar.take<double2>(2 * n);
  double* z = ar.take<double>(n);
  int64_t* m = ar.take<int64_t>(n);
  int* ovf = ar.take<int>(1);
  uint64_t* scratch = ar.take<uint64_t>((size_t)4 * level * n);
  HE_TRY(stage_reserve(c, sizeof(double) * n + 64));
  if (n_slots) {
    memcpy(c->h_stage, slots, sizeof(double) * n_slots);
    HE_CUDA(cudaMemcpyAsync(z, c->h_stage, sizeof(double) * n_slots, cudaMemcpyHostToDevice, c->stream));
  }
  HE_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c->stream));
  HE_TRY(encode_dev(c, z, n_slots, scale, m, fft, ovf));
  HE_TRY(encrypt_dev(c, m, level, use_sk, cid, out, scratch));
  HE_CUDA(cudaMemcpyAsync(c->h_stage, ovf, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  int flag = 0;
  memcpy(&flag, c->h_stage, sizeof(int));
  if (flag) return fail(HE_EINVAL, "encoded coefficient beyond int64");
  out->scale = scale;
  return HE_OK;
}

int he_decrypt_poly(he_ctx* c, const he_ct* ct, double* coeffs_out) {
  if (!c || !coeffs_out) return fail(HE_EINVAL, "he_decrypt_poly: null argument");
  HE_TRY(check_ct(c, ct, "he_decrypt_poly"));
  const size_t n = c->n;
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * ct->level * n + sizeof(double) * n + 4096));
  Arena ar = arena(c);
  uint64_t* m = ar.take<uint64_t>((size_t)ct->level * n);
  double* d = ar.take<double>(n);
  HE_TRY(decrypt_dev(c, ct, m, d));
  HE_TRY(stage_reserve(c, sizeof(double) * n));
  HE_CUDA(cudaMemcpyAsync(c->h_stage, d, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(coeffs_out, c->h_stage, sizeof(double) * n);
  return HE_OK;
}

int he_decrypt_decode(he_ctx* c, const he_ct* ct, double* slots_out, size_t n_slots) {
  if (!c || (!slots_out && n_slots)) return fail(HE_EINVAL, "he_decrypt_decode: null argument");
  HE_TRY(check_ct(c, ct, "he_decrypt_decode"));
  const size_t n = c->n;
  if (n_slots > n / 2) return fail(HE_EINVAL, "more slots than N/2");
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * ct->level * n + sizeof(double) * 2 * n + sizeof(double2) * 2 * n + 8192));
  Arena ar = arena(c);
  uint64_t* m = ar.take<uint64_t>((size_t)ct->level * n);
  double* d = ar.take<double>(n);
  double* re = ar.take<double>(n);
  double2* fft = ar.take<double2>(2 * n);
  HE_TRY(decrypt_dev(c, ct, m, d));
  HE_TRY(decode_dev(c, d, ct->scale, re, n_slots, fft));
  HE_TRY(stage_reserve(c, sizeof(double) * n));
  HE_CUDA(cudaMemcpyAsync(c->h_stage, re, sizeof(double) * n_slots, cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  memcpy(slots_out, c->h_stage, sizeof(double) * n_slots);
  return HE_OK;
}

int he_ct_alloc(he_ctx* c, uint32_t cap, he_ct** out) {
  if (!c || !out) return fail(HE_EINVAL, "he_ct_alloc: null argument");
  *out = nullptr;
  if (cap < 1 || cap > (uint32_t)c->L) return fail(HE_EINVAL, "he_ct_alloc: capacity outside [1, L]");
  he_ct* h = new he_ct();
  const size_t bytes = sizeof(uint64_t) * 2 * (size_t)cap * c->n;
  if (cudaMalloc(&h->data, bytes) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(HE_ENOMEM, "he_ct_alloc: device memory");
  }
  h->level = 0;
  h->cap = cap;
  h->scale = 0.0;
  *out = h;
  return HE_OK;
}

int he_ct_free(he_ct* ct) {
  if (!ct) return HE_OK;
  // the buffer may still be in use by work queued on any stream
  cudaError_t e = cudaDeviceSynchronize();
  cudaFree(ct->data);
  delete ct;
  return e == cudaSuccess ? HE_OK : fail(HE_ECUDA, std::string("he_ct_free: ") + cudaGetErrorString(e));
}

int he_ct_export(he_ctx* c, const he_ct* ct, uint64_t* host, size_t cap_words) {
  if (!c || !host) return fail(HE_EINVAL, "he_ct_export: null argument");
  HE_TRY(check_ct(c, ct, "he_ct_export"));
  const size_t lw = (size_t)ct->level * c->n;
  if (cap_words < 2 * lw) return fail(HE_EINVAL, "he_ct_export: host buffer too small");
  for (int p = 0; p < 2; ++p)
    HE_CUDA(cudaMemcpyAsync(host + p * lw, ct->data + (size_t)p * ct->cap * c->n, sizeof(uint64_t) * lw,
                            cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  return HE_OK;
}

int he_ct_import(he_ctx* c, const uint64_t* host, uint32_t level, double scale, he_ct* out) {
  if (!c || !host) return fail(HE_EINVAL, "he_ct_import: null argument");
  HE_TRY(check_out(c, out, level, "he_ct_import"));
  const size_t lw = (size_t)level * c->n;
  for (int p = 0; p < 2; ++p)
    HE_CUDA(cudaMemcpyAsync(out->data + (size_t)p * out->cap * c->n, host + p * lw, sizeof(uint64_t) * lw,
                            cudaMemcpyHostToDevice, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_ct_import_batch(he_ctx* c, const uint64_t* host, uint32_t level, double scale, he_ct* out, size_t count) {
  if (!c || !host || !out) return fail(HE_EINVAL, "he_ct_import_batch: null argument");
  const size_t lw = (size_t)level * c->n;
  for (size_t i = 0; i < count; ++i) HE_TRY(check_out(c, &out[i], level, "he_ct_import_batch"));
  // one copy per run of polynomials that are contiguous on the device too
  // (full-capacity ciphertexts back to back, as in a uniform batch)
  size_t run_src = 0, run_len = 0;
  uint64_t* run_dst = nullptr;
  for (size_t i = 0; i < count; ++i)
    for (int p = 0; p < 2; ++p) {
      uint64_t* dst = out[i].data + (size_t)p * out[i].cap * c->n;
      const size_t src = (i * 2 + p) * lw;
      if (run_dst && dst == run_dst + run_len && src == run_src + run_len) {
        run_len += lw;
        continue;
      }
      if (run_dst)
        HE_CUDA(cudaMemcpyAsync(run_dst, host + run_src, sizeof(uint64_t) * run_len, cudaMemcpyHostToDevice,
                                c->stream));
      run_dst = dst;
      run_src = src;
      run_len = lw;
    }
  if (run_dst)
    HE_CUDA(cudaMemcpyAsync(run_dst, host + run_src, sizeof(uint64_t) * run_len, cudaMemcpyHostToDevice, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  for (size_t i = 0; i < count; ++i) {
    out[i].level = level;
    out[i].scale = scale;
  }
  return HE_OK;
}

int he_ct_export_batch(he_ctx* c, const he_ct* cts, size_t count, uint64_t* host, size_t cap_words) {
  if (!c || !host || !cts) return fail(HE_EINVAL, "he_ct_export_batch: null argument");
  size_t off = 0;
  for (size_t i = 0; i < count; ++i) {
    HE_TRY(check_ct(c, &cts[i], "he_ct_export_batch"));
    off += 2 * (size_t)cts[i].level * c->n;
  }
  if (off > cap_words) return fail(HE_EINVAL, "he_ct_export_batch: host buffer too small");
  // one copy per run of polynomials that are contiguous on the device too
  off = 0;
  size_t run_dst = 0, run_len = 0;
  const uint64_t* run_src = nullptr;
  for (size_t i = 0; i < count; ++i) {
    const size_t lw = (size_t)cts[i].level * c->n;
    for (int p = 0; p < 2; ++p) {
      const uint64_t* src = cts[i].data + (size_t)p * cts[i].cap * c->n;
      if (run_src && src == run_src + run_len && off == run_dst + run_len) {
        run_len += lw;
      } else {
        if (run_src)
          HE_CUDA(cudaMemcpyAsync(host + run_dst, run_src, sizeof(uint64_t) * run_len, cudaMemcpyDeviceToHost,
                                  c->stream));
        run_src = src;
        run_dst = off;
        run_len = lw;
      }
      off += lw;
    }
  }
  if (run_src)
    HE_CUDA(cudaMemcpyAsync(host + run_dst, run_src, sizeof(uint64_t) * run_len, cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  return HE_OK;
}

static int addsub(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out, int op) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_add"));
  HE_TRY(check_ct(c, b, "he_add"));
  if (!scales_match(a->scale, b->scale)) return fail(HE_ESCALE, "operand scales differ");
  const uint32_t level = std::min(a->level, b->level);
  HE_TRY(check_out(c, out, level, "he_add"));
  const double scale = a->scale;
  HE_TRY(addsub_batch(c, one(a), one(b), one(out), op, level, 1));
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_add(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out) { return addsub(c, a, b, out, 0); }
int he_sub(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out) { return addsub(c, a, b, out, 1); }

int he_sum(he_ctx* c, const he_ct* a, size_t count, he_ct* out) {
  if (!c || !a || count == 0) return fail(HE_EINVAL, "he_sum: null argument or no ciphertext");
  uint32_t level = (uint32_t)c->L;
  for (size_t i = 0; i < count; ++i) {
    HE_TRY(check_ct(c, &a[i], "he_sum"));
    if (!scales_match(a[i].scale, a[0].scale)) return fail(HE_ESCALE, "he_sum: scales differ");
    level = std::min(level, a[i].level);
  }
  HE_TRY(check_out(c, out, level, "he_sum"));
  for (size_t i = 1; i < count; ++i)
    if (a[i].data == out->data) return fail(HE_EINVAL, "he_sum: out may alias only the first input");
  const double scale = a[0].scale;
  if (a[0].data != out->data) HE_TRY(copy_batch(c, one(&a[0]), one(out), level, 1));
  if (count > 1) {
    CtBatch rest;
    if (uniform_view(a + 1, count - 1, &rest)) {
      HE_TRY(accumulate_batch(c, rest, (uint32_t)(count - 1), one(out), level));
    } else {
      for (size_t i = 1; i < count; ++i) HE_TRY(addsub_batch(c, one(out), one(&a[i]), one(out), 0, level, 1));
    }
  }
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_drop_level(he_ctx* c, const he_ct* a, uint32_t level, he_ct* out) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_drop_level"));
  if (level < 1 || level > a->level) return fail(HE_EINVAL, "he_drop_level: bad target level");
  HE_TRY(check_out(c, out, level, "he_drop_level"));
  const double scale = a->scale;
  if (out->data != a->data || out->cap != a->cap) HE_TRY(copy_batch(c, one(a), one(out), level, 1));
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_mul_const(he_ctx* c, const he_ct* a, double value, double value_scale, he_ct* out) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_mul_const"));
  HE_TRY(check_out(c, out, a->level, "he_mul_const"));
  const double v = value * value_scale;
  if (!(fabs(v) < 9.2e18)) return fail(HE_EINVAL, "constant beyond int64");
  const uint32_t level = a->level;
  const double scale = a->scale * value_scale;
  HE_TRY(mul_int_batch(c, one(a), one(out), (int64_t)llround(v), level, 1));
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_add_const(he_ctx* c, const he_ct* a, double value, he_ct* out) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_add_const"));
  HE_TRY(check_out(c, out, a->level, "he_add_const"));
  const double v = value * a->scale;
  if (!(fabs(v) < 9.2e18)) return fail(HE_EINVAL, "constant beyond int64");
  const uint32_t level = a->level;
  const double scale = a->scale;
  HE_TRY(add_int_batch(c, one(a), one(out), (int64_t)llround(v), level, 1));
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_mul_plain(he_ctx* c, const he_ct* a, const int64_t* coeffs, double pt_scale, he_ct* out) {
  if (!c || !coeffs) return fail(HE_EINVAL, "he_mul_plain: null argument");
  HE_TRY(check_ct(c, a, "he_mul_plain"));
  HE_TRY(check_out(c, out, a->level, "he_mul_plain"));
  const size_t n = c->n;
  const uint32_t level = a->level;
  const double scale = a->scale * pt_scale;
  HE_TRY(ws_reserve(c, sizeof(int64_t) * n + sizeof(uint64_t) * level * n + 4096));
  Arena ar = arena(c);
  int64_t* m = ar.take<int64_t>(n);
  HE_TRY(stage_reserve(c, sizeof(int64_t) * n));
  memcpy(c->h_stage, coeffs, sizeof(int64_t) * n);
  HE_CUDA(cudaMemcpyAsync(m, c->h_stage, sizeof(int64_t) * n, cudaMemcpyHostToDevice, c->stream));
  HE_TRY(mul_plain_dev(c, one(a), m, one(out), level, 1, ar));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  out->level = level;
  out->scale = scale;
  return HE_OK;
}

int he_rescale(he_ctx* c, const he_ct* a, he_ct* out) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_rescale"));
  if (a->level < 2) return fail(HE_ELEVEL, "he_rescale: one limb left");
  HE_TRY(check_out(c, out, a->level - 1, "he_rescale"));
  const uint32_t level = a->level;
  const double scale = a->scale / (double)c->q[level - 1];
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * rescale_words(c, level, 1) + 4096));
  Arena ar = arena(c);
  HE_TRY(rescale_batch(c, one(a), level, 1, one(out), ar));
  out->level = level - 1;
  out->scale = scale;
  return HE_OK;
}

// Multiplications of `count` pairs (uniform views), chunked by the scratch budget.
static int mul_chunks(he_ctx* c, CtBatch A, CtBatch B, CtBatch O, uint32_t level, size_t count, bool rescale) {
  const size_t per = mul_words(c, level, 1, rescale) * sizeof(uint64_t);
  size_t chunk = std::max<size_t>(1, c->chunk_bytes / per);
  chunk = std::min(chunk, count);
  HE_TRY(ws_reserve(c, mul_words(c, level, (uint32_t)chunk, rescale) * sizeof(uint64_t) + 8192));
  for (size_t i0 = 0; i0 < count; i0 += chunk) {
    const uint32_t m = (uint32_t)std::min(chunk, count - i0);
    CtBatch a = A, b = B, o = O;
    a.base += i0 * A.stride;
    b.base += i0 * B.stride;
    o.base += i0 * O.stride;
    Arena ar = arena(c);
    HE_TRY(mul_relin_batch(c, a, b, level, m, o, rescale, ar));
  }
  return HE_OK;
}

static int mul_common(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out, bool rescale) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_mul"));
  HE_TRY(check_ct(c, b, "he_mul"));
  const uint32_t level = std::min(a->level, b->level);
  if (rescale && level < 2) return fail(HE_ELEVEL, "multiplication needs two limbs to rescale");
  HE_TRY(check_out(c, out, rescale ? level - 1 : level, "he_mul"));
  const double scale = rescale ? a->scale * b->scale / (double)c->q[level - 1] : a->scale * b->scale;
  HE_TRY(mul_chunks(c, one(a), one(b), one(out), level, 1, rescale));
  out->level = rescale ? level - 1 : level;
  out->scale = scale;
  return HE_OK;
}

int he_mul_relin_rescale(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out) {
  return mul_common(c, a, b, out, true);
}

int he_mul_relin(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out) { return mul_common(c, a, b, out, false); }

int he_mul_relin_rescale_batch(he_ctx* c, const he_ct* a, const he_ct* b, he_ct* out, size_t count) {
  if (!c || !a || !b || !out) return fail(HE_EINVAL, "he_mul_relin_rescale_batch: null argument");
  if (count == 0) return HE_OK;
  for (size_t i = 0; i < count; ++i) {
    HE_TRY(check_ct(c, &a[i], "he_mul_relin_rescale_batch"));
    HE_TRY(check_ct(c, &b[i], "he_mul_relin_rescale_batch"));
    if (a[i].level != a[0].level || b[i].level != a[0].level)
      return fail(HE_EINVAL, "batched operands must share one level");
  }
  const uint32_t level = a[0].level;
  if (level < 2) return fail(HE_ELEVEL, "multiplication needs two limbs to rescale");
  for (size_t i = 0; i < count; ++i) HE_TRY(check_out(c, &out[i], level - 1, "he_mul_relin_rescale_batch"));
  CtBatch A, B, O;
  if (uniform_view(a, count, &A) && uniform_view(b, count, &B) && uniform_view(out, count, &O)) {
    HE_TRY(mul_chunks(c, A, B, O, level, count, true));
  } else {
    for (size_t i = 0; i < count; ++i) HE_TRY(mul_chunks(c, one(&a[i]), one(&b[i]), one(&out[i]), level, 1, true));
  }
  const double ql = (double)c->q[level - 1];
  for (size_t i = 0; i < count; ++i) {
    out[i].scale = a[i].scale * b[i].scale / ql;
    out[i].level = level - 1;
  }
  return HE_OK;
}

static int rot_chunks(he_ctx* c, CtBatch A, CtBatch O, uint32_t level, size_t count, uint64_t gal) {
  const size_t per = rot_words(c, level, 1) * sizeof(uint64_t);
  size_t chunk = std::max<size_t>(1, c->chunk_bytes / per);
  chunk = std::min(chunk, count);
  HE_TRY(ws_reserve(c, rot_words(c, level, (uint32_t)chunk) * sizeof(uint64_t) + 8192));
  for (size_t i0 = 0; i0 < count; i0 += chunk) {
    const uint32_t m = (uint32_t)std::min(chunk, count - i0);
    CtBatch a = A, o = O;
    a.base += i0 * A.stride;
    o.base += i0 * O.stride;
    Arena ar = arena(c);
    HE_TRY(rotate_batch(c, a, level, m, gal, o, ar));
  }
  return HE_OK;
}

int he_rotate(he_ctx* c, const he_ct* a, int32_t steps, he_ct* out) { return he_rotate_batch(c, a, steps, out, 1); }

int he_rotate_batch(he_ctx* c, const he_ct* a, int32_t steps, he_ct* out, size_t count) {
  if (!c || !a || !out) return fail(HE_EINVAL, "he_rotate: null argument");
  if (count == 0) return HE_OK;
  for (size_t i = 0; i < count; ++i) {
    HE_TRY(check_ct(c, &a[i], "he_rotate"));
    if (a[i].level != a[0].level) return fail(HE_EINVAL, "batched operands must share one level");
    HE_TRY(check_out(c, &out[i], a[i].level, "he_rotate"));
  }
  const uint32_t level = a[0].level;
  const uint64_t gal = h_galois_elt(c->log_n, steps);
  if (gal != 1 && !galois_key(c, gal)) return fail(HE_ENOKEY, "no Galois key for this rotation");
  CtBatch A, O;
  if (gal == 1) {
    for (size_t i = 0; i < count; ++i)
      if (out[i].data != a[i].data) HE_TRY(copy_batch(c, one(&a[i]), one(&out[i]), level, 1));
  } else if (uniform_view(a, count, &A) && uniform_view(out, count, &O)) {
    HE_TRY(rot_chunks(c, A, O, level, count, gal));
  } else {
    for (size_t i = 0; i < count; ++i) HE_TRY(rot_chunks(c, one(&a[i]), one(&out[i]), level, 1, gal));
  }
  for (size_t i = 0; i < count; ++i) {
    out[i].level = level;
    out[i].scale = a[i].scale;
  }
  return HE_OK;
}

static int rotsum_chunks(he_ctx* c, CtBatch A, CtBatch O, uint32_t level, size_t count, const uint64_t* gals,
                         uint32_t nrot) {
  const size_t per = rotsum_words(c, level, 1) * sizeof(uint64_t);
  size_t chunk = std::max<size_t>(1, c->chunk_bytes / per);
  chunk = std::min(chunk, count);
  HE_TRY(ws_reserve(c, rotsum_words(c, level, (uint32_t)chunk) * sizeof(uint64_t) + 8192));
  for (size_t i0 = 0; i0 < count; i0 += chunk) {
    const uint32_t m = (uint32_t)std::min(chunk, count - i0);
    CtBatch a = A, o = O;
    a.base += i0 * A.stride;
    o.base += i0 * O.stride;
    Arena ar = arena(c);
    HE_TRY(rotsum_batch(c, a, level, m, gals, nrot, o, ar));
  }
  return HE_OK;
}

int he_rotate_sum(he_ctx* c, const he_ct* a, const int32_t* steps, uint32_t nsteps, he_ct* out) {
  return he_rotate_sum_batch(c, a, steps, nsteps, out, 1);
}

int he_rotate_sum_batch(he_ctx* c, const he_ct* a, const int32_t* steps, uint32_t nsteps, he_ct* out,
                        size_t count) {
  if (!c || !a || !out || !steps) return fail(HE_EINVAL, "he_rotate_sum: null argument");
  if (nsteps < 1 || nsteps > HE_MAX_ROT) return fail(HE_EINVAL, "he_rotate_sum: 1 to 16 steps");
  if (count == 0) return HE_OK;
  for (size_t i = 0; i < count; ++i) {
    HE_TRY(check_ct(c, &a[i], "he_rotate_sum"));
    if (a[i].level != a[0].level) return fail(HE_EINVAL, "batched operands must share one level");
    HE_TRY(check_out(c, &out[i], a[i].level, "he_rotate_sum"));
  }
  const uint32_t level = a[0].level;
  uint64_t gals[HE_MAX_ROT];
  for (uint32_t r = 0; r < nsteps; ++r) {
    gals[r] = h_galois_elt(c->log_n, steps[r]);
    if (gals[r] == 1) return fail(HE_EINVAL, "he_rotate_sum: a rotation by 0 slots");
    if (!galois_key(c, gals[r])) return fail(HE_ENOKEY, "no Galois key for this rotation");
  }
  // out[i] may be a[i] (then through a copy of the input); no other overlap
  bool overlap = false;
  for (size_t i = 0; i < count; ++i)
    for (size_t k = 0; k < count; ++k) {
      const char* a_lo = (const char*)a[i].data;
      const char* a_hi = a_lo + sizeof(uint64_t) * 2 * (size_t)a[i].cap * c->n;
      const char* o_lo = (const char*)out[k].data;
      const char* o_hi = o_lo + sizeof(uint64_t) * 2 * (size_t)out[k].cap * c->n;
      if (o_hi <= a_lo || a_hi <= o_lo) continue;
      if (i != k) return fail(HE_EINVAL, "he_rotate_sum: an output overlaps another ciphertext's input");
      overlap = true;
    }
  CtBatch A, O;
  if (!overlap && uniform_view(a, count, &A) && uniform_view(out, count, &O)) {
    HE_TRY(rotsum_chunks(c, A, O, level, count, gals, nsteps));
  } else {
    uint64_t* tmp = nullptr;
    if (cudaMalloc(&tmp, sizeof(uint64_t) * 2 * (size_t)level * c->n) != cudaSuccess) {
      cudaGetLastError();
      return fail(HE_ENOMEM, "he_rotate_sum: copy of the input");
    }
    int rc = HE_OK;
    const CtBatch T{tmp, 0, level, 0};
    for (size_t i = 0; i < count && rc == HE_OK; ++i) {
      rc = copy_batch(c, one(&a[i]), T, level, 1);
      if (rc == HE_OK) rc = rotsum_chunks(c, T, one(&out[i]), level, 1, gals, nsteps);
    }
    cudaStreamSynchronize(c->stream);
    cudaFree(tmp);
    HE_TRY(rc);
  }
  for (size_t i = 0; i < count; ++i) {
    out[i].level = level;
    out[i].scale = a[i].scale;
  }
  return HE_OK;
}

int he_refresh(he_ctx* c, const he_ct* a, uint32_t level, double out_scale, uint32_t cid, he_ct* out) {
  if (!c) return fail(HE_EINVAL, "null context");
  HE_TRY(check_ct(c, a, "he_refresh"));
  HE_TRY(check_out(c, out, level, "he_refresh"));
  const size_t n = c->n;
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * a->level * n + sizeof(double) * 2 * n + sizeof(double2) * 2 * n +
                           sizeof(int64_t) * n + sizeof(uint64_t) * 4 * level * n + 16384));
  Arena ar = arena(c);
  uint64_t* m = ar.take<uint64_t>((size_t)a->level * n);
  double* d = ar.take<double>(n);
  double* re = ar.take<double>(n);
  double2* fft = ar.take<double2>(2 * n);
  int64_t* coeffs = ar.take<int64_t>(n);
  int* ovf = ar.take<int>(1);
  uint64_t* scratch = ar.take<uint64_t>((size_t)4 * level * n);
  // key holder: decrypt and decode ...
  HE_TRY(decrypt_dev(c, a, m, d));
  HE_TRY(decode_dev(c, d, a->scale, re, n / 2, fft));
  // ... re-encode and encrypt at the requested level
  HE_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c->stream));
  HE_TRY(encode_dev(c, re, n / 2, out_scale, coeffs, fft, ovf));
  HE_TRY(encrypt_dev(c, coeffs, level, 0, cid, out, scratch));
  HE_TRY(stage_reserve(c, 64));
  HE_CUDA(cudaMemcpyAsync(c->h_stage, ovf, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  HE_CUDA(cudaStreamSynchronize(c->stream));
  int flag = 0;
  memcpy(&flag, c->h_stage, sizeof(int));
  if (flag) return fail(HE_EINVAL, "refresh: encoded coefficient beyond int64");
  out->level = level;
  out->scale = out_scale;
  return HE_OK;
}

int he_ntt(he_ctx* c, uint64_t* data, uint32_t npolys, uint64_t poly_stride, uint32_t nl, uint32_t prime0,
           int inverse) {
  if (!c || !data) return fail(HE_EINVAL, "he_ntt: null argument");
  if (((uintptr_t)data & 7) || npolys == 0) return fail(HE_EINVAL, "he_ntt: misaligned data or no polynomials");
  if (prime0 + nl > (uint32_t)c->np || nl == 0) return fail(HE_EINVAL, "he_ntt: limbs beyond the primes");
  PolyBatch b;
  b.src = data;
  b.dst = data;
  b.src_stride = b.dst_stride = poly_stride;
  b.npolys = npolys;
  b.nl = nl;
  b.limb0 = prime0;
  b.level = (uint32_t)c->np;  // identity map: limb t -> prime t
  b.skip_alpha = 0;
  b.skip_beta = 1;
  return inverse ? ntt_inverse(c, b) : ntt_forward(c, b);
}

int he_keyswitch(he_ctx* c, const uint64_t* d, uint32_t level, uint64_t galois, uint64_t* out0, uint64_t* out1) {
  if (!c || !d || !out0 || !out1) return fail(HE_EINVAL, "he_keyswitch: null argument");
  if (!aligned16(d) || !aligned16(out0) || !aligned16(out1)) return fail(HE_EINVAL, "he_keyswitch: pointers must be 16-byte aligned");
  if (level < 1 || level > (uint32_t)c->L) return fail(HE_EINVAL, "he_keyswitch: bad level");
  const uint64_t* key = galois ? galois_key(c, galois) : c->d_rlk;
  if (!key) return fail(HE_ENOKEY, "he_keyswitch: no key for this Galois element");
  const size_t n = c->n;
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * (ks_words(c, level, 1) + 2 * level * n) + 8192));
  Arena ar = arena(c);
  uint64_t* o = ar.take<uint64_t>((size_t)2 * level * n);
  CtBatch O{o, 0, level, 0};
  HE_TRY(keyswitch_batch(c, d, 0, level, 1, key, O, 0, O, ar));
  HE_CUDA(cudaMemcpyAsync(out0, o, sizeof(uint64_t) * level * n, cudaMemcpyDeviceToDevice, c->stream));
  HE_CUDA(cudaMemcpyAsync(out1, o + (size_t)level * n, sizeof(uint64_t) * level * n, cudaMemcpyDeviceToDevice,
                          c->stream));
  return HE_OK;
}

int he_moddown(he_ctx* c, const uint64_t* acc, uint32_t level, const he_ct* d01, he_ct* out) {
  if (!c || !acc) return fail(HE_EINVAL, "he_moddown: null argument");
  if (!aligned16(acc)) return fail(HE_EINVAL, "he_moddown: pointers must be 16-byte aligned");
  if (level < 1 || level > (uint32_t)c->L) return fail(HE_EINVAL, "he_moddown: bad level");
  const bool merged = d01 != nullptr;
  if (merged) {
    if (level < 2) return fail(HE_ELEVEL, "he_moddown: the merged rescale needs two limbs");
    if (!c->d_mdrs) return fail(HE_EINVAL, "he_moddown: no merged tables (more than 7 special primes)");
    HE_TRY(check_ct(c, d01, "he_moddown"));
    if (d01->level != level) return fail(HE_EINVAL, "he_moddown: d01 must be at the accumulator's level");
  }
  const uint32_t lt = merged ? level - 1 : level;
  HE_TRY(check_out(c, out, lt, "he_moddown"));
  const size_t n = c->n, nt = level + (size_t)c->alpha;
  HE_TRY(ws_reserve(c, sizeof(uint64_t) * (2 * nt * n + 4 * level * n) + 8192));
  Arena ar = arena(c);
  uint64_t* a = ar.take<uint64_t>(2 * nt * n);
  uint64_t* conv = ar.take<uint64_t>(2 * (size_t)level * n);
  if (!a || !conv) return fail(HE_ENOMEM, "he_moddown: scratch too small");
  HE_CUDA(cudaMemcpyAsync(a, acc, sizeof(uint64_t) * 2 * nt * n, cudaMemcpyDeviceToDevice, c->stream));
  const CtBatch add = merged ? one(d01) : CtBatch{nullptr, 0, 0, 0};
  HE_TRY(moddown_batch(c, a, conv, level, 1, add, merged ? 2 : 0, one(out), ar, 0, merged));
  out->level = lt;
  if (merged) out->scale = d01->scale;
  return HE_OK;
}

}  // extern "C"
