// he_internal.h -- host-side context of the RNS-CKKS worker library.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <atomic>
#include <map>
#include <string>
#include <vector>

#include "../../include/he_gb300.h"
#include "he_common.cuh"

namespace he {

// ---- status handling -------------------------------------------------------
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);

#define HE_CUDA(call)                                                              \
  do {                                                                             \
    cudaError_t e_ = (call);                                                       \
    if (e_ != cudaSuccess)                                                         \
      return ::he::fail(HE_ECUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

#define HE_TRY(call)             \
  do {                                \
    int rc_ = (call);                 \
    if (rc_ != HE_OK) return rc_;     \
  } while (0)

// cudaFuncSetAttribute (the dynamic shared memory a kernel may take) once per
// device for each kernel instance: `bits` is that instance's set of devices
// done, an atomic so that host threads first using a ring size at the same
// time do not race on it (a repeated call is harmless).
inline int set_smem_attr_once(std::atomic<unsigned long long>& bits, int device, const void* fn, size_t bytes) {
  if (device < 0 || device >= 64) return HE_OK;
  const unsigned long long m = 1ull << device;
  if (bits.load(std::memory_order_acquire) & m) return HE_OK;
  HE_CUDA(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  bits.fetch_or(m, std::memory_order_acq_rel);
  return HE_OK;
}

// ---- host number theory (params.cpp) ---------------------------------------
uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q);
uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t q);
uint64_t h_invmod(uint64_t a, uint64_t q);
bool h_is_prime(uint64_t n);
std::vector<uint64_t> h_ntt_primes(int bits, int log_n, int count, const std::vector<uint64_t>& skip);
uint64_t h_min_root(uint64_t q, int log_n);
uint64_t h_shoup(uint64_t w, uint64_t q);
int h_gauss_table(double sigma, uint64_t* T);
uint64_t h_galois_elt(int log_n, int32_t r);

// Per-(level, digit) basis-conversion constants for ModUp, laid out in one
// device buffer: for the digit's limbs i: inv (Shoup pair), then a row of
// (Q_j/q_i) mod p for every prime index p < np.
struct ModUpConst {
  uint32_t lo, cnt;  // digit limbs [lo, lo + cnt)
  size_t off;        // word offset of this table in d_modup
};

struct Workspace {
  void* ptr = nullptr;
  size_t size = 0;
};

struct ProfClass {
  uint64_t launches = 0;
  double work = 0.0, bytes = 0.0;
  double mac = 0.0;   // the part of work that is unreduced 128-bit multiply-accumulates
  double mac3 = 0.0;  // ... that is split products summed as three 64-bit sums (mac_split3)
  double bfly = 0.0;  // the part of work that is NTT butterflies
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
};

}  // namespace he

struct he_ctx {
  he_params prm;
  bool view = false;  // shares the tables and keys of another context (frees only its own state)
  int log_n = 0, n = 0, L = 0, alpha = 0, np = 0, beta = 0;
  std::vector<uint64_t> q;    // [np]: limbs then special primes
  std::vector<uint64_t> psi;  // [np]
  cudaStream_t stream = nullptr;
  int device = 0;
  size_t smem_per_sm = 228 * 1024;  // shared memory of one SM (queried at creation)

  // device tables
  PrimeDev* d_primes = nullptr;  // [np]
  uint64_t* d_tw = nullptr;      // [np][N] pairs (psi^brv(m), its Shoup companion)
  uint64_t* d_itw = nullptr;     // [np][N] pairs (psi^-brv(m), its Shoup companion)
  uint64_t* d_two64 = nullptr;   // [np] 2^64 mod q
  uint64_t* d_gauss = nullptr;   // Gaussian CDT
  int gK = 0;

  // ModUp constants per (level, digit): host index + device words
  std::vector<std::vector<he::ModUpConst>> modup;  // [level][digit]
  uint64_t* d_modup = nullptr;
  // ModDown: for special k: inv (Shoup pair) [alpha][2]; mat [alpha][L]; P^-1 mod q_t pair [L][2]
  uint64_t* d_moddown = nullptr;
  // Rescale: q_{l-1}^-1 mod q_t Shoup pairs [L][L][2]
  uint64_t* d_rescale = nullptr;
  uint64_t* d_rescale_md = nullptr;  // per dropped limb l: the ModDown tables with q_l as the one special prime
  size_t rescale_md_words = 0;       // words per l
  uint64_t* d_mdrs = nullptr;        // per level l: the ModDown tables dividing by P q_{l-1} (ModDown + rescale)
  size_t mdrs_words = 0;             // words per l
  // Garner (decryption CRT): [L] Shoup pairs of (q_0..q_{i-1})^-1 mod q_i, then
  // [L][L] prefix products (q_0..q_{i'-1}) mod q_i
  uint64_t* d_garner = nullptr;
  size_t chunk_bytes = (size_t)1 << 34;  // scratch budget of one batched operation (16 GiB)
  uint32_t lr_chunk = 0;                 // data ciphertexts per chunk of the LR step (0: from the budget)
  bool ntt_generic = false;              // force the runtime-shaped NTT kernel (tuning)
  int ntt_shape = 0;                     // NTT tile shapes: 0, 1 or 2 (ntt2.cu)
  uint32_t ntt_pb_max = 8;               // polynomials of one limb per NTT CTA, at most
  uint32_t ks_ct = 0;                    // ciphertexts per key-product CTA in closed stages (0: most that fit)
  std::map<std::string, cudaGraphExec_t> graphs;  // captured multi-worker steps
  std::vector<uint64_t> P_mod_q;  // [L] P mod q_t (host)

  // keys (evaluation form)
  uint64_t* d_s = nullptr;    // [np][N]
  uint64_t* d_pk = nullptr;   // [2][L][N] (b, a)
  uint64_t* d_rlk = nullptr;  // [beta][2][np][N]
  std::map<uint64_t, uint64_t*> gal;  // Galois element -> [beta][2][np][N]
  // encoded 0/1 masks of the logistic-regression step, per (g, scale)
  std::map<std::pair<uint32_t, double>, int64_t*> lr_masks;

  he::Workspace ws;
  uint64_t ws_requests = 0;  // calls of ws_reserve on this context (he_ctx_workspace)
  bool prof_on = false;
  std::map<std::string, he::ProfClass> prof;
  uint64_t* h_stage = nullptr;  // pinned staging (host <-> device)
  size_t h_stage_size = 0;
  // host-input step: device copy of the inputs, a copy stream and one event per
  // piece of data ciphertexts; the step waits for a piece before its chunk
  he::Workspace io;
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> io_events;
  size_t io_piece = 0;             // data ciphertexts per copied piece (0: no pipelined input)
  size_t io_first_chunk = 0;       // data ciphertexts of the step's first chunk (0: a full chunk)
  // timing of the last host-input step: its copies (copy stream) and its
  // first chunk's arithmetic (step stream); sizes the next first chunk
  cudaEvent_t io_time[4] = {nullptr, nullptr, nullptr, nullptr};
  size_t io_timed_nZ = 0, io_timed_first = 0;  // ciphertexts the events cover (0: none)
  size_t io_pieces_waited = 0;     // pieces the step's stream already waits for

  size_t key_words() const { return (size_t)beta * 2 * np * n; }
};

namespace he {

// ---- kernel timing (prof.cu) ------------------------------------------------------
// RAII bracket of one launch: adds `work` (algorithmic units) and `bytes`
// (algorithmic DRAM bytes) to kernel class `name` when timing is enabled.
class ProfScope {
 public:
  ProfScope(he_ctx* c, const char* name, double work, double bytes, double mac = 0.0, double bfly = 0.0,
            double mac3 = 0.0);
  ~ProfScope();

 private:
  he_ctx* c_;
  cudaEvent_t stop_ = nullptr;
};
void prof_clear(he_ctx* c);
// While one of these lives, launches on this host thread are not timed
// (ProfScope records nothing), whatever the context's setting: for entry
// points that must create no CUDA objects, without touching shared state.
class ProfSuppress {
 public:
  ProfSuppress();
  ~ProfSuppress();

 private:
  bool prev_;
};

// ---- workspace ----------------------------------------------------------------
int ws_reserve(he_ctx* c, size_t bytes);  // may reallocate (synchronises first)
// A context sharing `base`'s tables and keys with its own stream and workspace.
he_ctx* ctx_view(he_ctx* base, cudaStream_t stream);
void ctx_destroy(he_ctx* c);
int stage_reserve(he_ctx* c, size_t bytes);

// ---- NTT (ntt.cu) -------------------------------------------------------------
// A batch of npolys polynomials: polynomial p's transformed limbs are
// limb0 .. limb0+nl-1, the first of them at src + p*src_stride (words) and
// the others N words apart (likewise dst).  Limb t maps to prime t when
// t < level, else to the special prime L + (t - level).  When skip_alpha > 0,
// polynomial p belongs to digit j = p % skip_beta and its limbs
// [j*skip_alpha, min((j+1)*skip_alpha, level)) are left untouched.
struct PolyBatch {
  const uint64_t* src;
  uint64_t* dst;
  uint64_t src_stride, dst_stride;
  uint32_t npolys, nl, limb0, level;
  uint32_t skip_alpha, skip_beta;
  uint64_t gal = 0;  // inverse transforms: read the source through this automorphism (0: none)
};
int ntt_forward(he_ctx* c, const PolyBatch& b);
int ntt_inverse(he_ctx* c, const PolyBatch& b);

}  // namespace he
