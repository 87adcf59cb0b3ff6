// he_ops.h -- batched ciphertext operations composed from the kernels.
#pragma once
#include <vector>

#include "he_internal.h"
#include "he_kernels.h"

namespace he {

unsigned grid_for(size_t work);

// Bump allocator over a caller-reserved device region (256-byte aligned).
struct Arena {
  char* base = nullptr;
  size_t size = 0, off = 0;
  template <class T>
  T* take(size_t count) {
    const size_t bytes = (count * sizeof(T) + 255) & ~(size_t)255;
    if (off + bytes > size) return nullptr;
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

int build_tables(he_ctx* c);
int keygen(he_ctx* c, const std::vector<int32_t>& rots);

// codec.cu / keys.cu (scratch passed explicitly)
int encode_dev(he_ctx* c, const double* d_z, size_t n_slots, double scale, int64_t* d_out,
               double2* scratch, int* d_ovf);
int decrypt_dev(he_ctx* c, const he_ct* ct, uint64_t* m, double* d_coeffs);
int decode_dev(he_ctx* c, const double* d_m, double scale, double* d_re, size_t n_slots,
               double2* scratch);
int encrypt_dev(he_ctx* c, const int64_t* d_m, uint32_t level, int use_sk, uint32_t cid, he_ct* out,
                uint64_t* scratch);

// Scratch words needed by one key switch / multiplication / rotation / rescale
// of `count` ciphertexts at `level`.
size_t ks_words(const he_ctx* c, uint32_t level, uint32_t count);
size_t mul_words(const he_ctx* c, uint32_t level, uint32_t count, bool rescale);
size_t rot_words(const he_ctx* c, uint32_t level, uint32_t count);
size_t rescale_words(const he_ctx* c, uint32_t level, uint32_t count);

// add_mode: 0 none, 1 add to part 0 only, 2 add to both parts.  gal != 0:
// d and the addend are read through the automorphism X -> X^gal (fused
// kernels only; the output must not overlap them).
// merged: divide P * add + (the inner products) by P q_{level-1} with one
// rounding (the ModDown and the rescale of a multiplication; add_mode 2, add
// = (d0, d1), out has level - 1 limbs).
int keyswitch_batch(he_ctx* c, const uint64_t* d, uint64_t d_stride, uint32_t level, uint32_t count,
                    const uint64_t* evk, CtBatch add, int add_mode, CtBatch out, Arena& ar, uint64_t gal = 0,
                    bool merged = false);
// The key switch's ModDown alone: acc (count x [2][level + alpha][N],
// evaluation form over Q_level and P; its dropped limbs are overwritten)
// divided by P with rounding (merged: P add + acc divided by P q_{level-1}),
// conv (count x [2][level][N]) as scratch; add_mode and gal as above.
int moddown_batch(he_ctx* c, uint64_t* acc, uint64_t* conv, uint32_t level, uint32_t count, CtBatch add,
                  int add_mode, CtBatch out, Arena& ar, uint64_t gal, bool merged);
// Whether N has compiled shapes for the fused key-switching kernels.
inline bool ks_fusable(const he_ctx* c) { return !c->ntt_generic && c->log_n >= 12 && c->log_n <= 16; }
int rescale_batch(he_ctx* c, CtBatch in, uint32_t level, uint32_t count, CtBatch out, Arena& ar);
int mul_relin_batch(he_ctx* c, CtBatch A, CtBatch B, uint32_t level, uint32_t count, CtBatch out,
                    bool rescale, Arena& ar);
int rotate_batch(he_ctx* c, CtBatch A, uint32_t level, uint32_t count, uint64_t gal, CtBatch out,
                 Arena& ar);
int addsub_batch(he_ctx* c, CtBatch A, CtBatch B, CtBatch O, int op, uint32_t level, uint32_t count);
// out = A + sum_r rotate(A, gals[r]) (1 <= nrot <= HE_MAX_ROT), one hoisted
// decomposition and one ModDown; out must not overlap A.
int rotsum_batch(he_ctx* c, CtBatch A, uint32_t level, uint32_t count, const uint64_t* gals, uint32_t nrot,
                 CtBatch out, Arena& ar);
size_t rotsum_words(const he_ctx* c, uint32_t level, uint32_t count);
int mul_int_batch(he_ctx* c, CtBatch A, CtBatch O, int64_t k, uint32_t level, uint32_t count);
int add_int_batch(he_ctx* c, CtBatch A, CtBatch O, int64_t k, uint32_t level, uint32_t count);
int copy_batch(he_ctx* c, CtBatch A, CtBatch O, uint32_t level, uint32_t count);
// acc += sum_i in[i] over `count` ciphertexts.
int accumulate_batch(he_ctx* c, CtBatch in, uint32_t count, CtBatch acc, uint32_t level);
// acc ([3][level][N]) += sum_i tensor(A[i], B[i]) over `count` pairs.
int tensor_acc_batch(he_ctx* c, CtBatch A, CtBatch B, uint32_t count, uint64_t* acc, uint32_t level);
// out = rescale(relinearise(D)) for three-part D (count x [3][level][N] at d_stride).
int relin_rescale_batch(he_ctx* c, uint64_t* D, uint64_t d_stride, uint32_t level, uint32_t count, CtBatch out,
                        Arena& ar);

const uint64_t* galois_key(const he_ctx* c, uint64_t gal);
bool uniform_view(const he_ct* a, size_t count, CtBatch* out);
// The logistic-regression step (infer = false) or inference (true) for
// several workers; see he_lr_gradient_step_workers.
int lr_entry(he_ctx* c, const he_lr_shard* shards, size_t count, const he_lr_config* cfg, uint32_t refresh_level,
             int flags, bool infer);
// Workspace bytes lr_entry reserves for shards of these shapes (circuit input
// level l0, data ciphertexts nZ, weights refreshed first or not).
struct LrShape {
  uint32_t l0;
  size_t nZ;
  bool refresh;
};
size_t lr_ws_bytes(he_ctx* c, const LrShape* sh, size_t count, uint32_t refresh_level);
// Bytes ws_reserve allocates for a request of `bytes` (headroom included).
size_t ws_alloc_bytes(size_t bytes);
int mul_plain_dev(he_ctx* c, CtBatch A, const int64_t* d_coeffs, CtBatch O, uint32_t level, uint32_t count,
                  Arena& ar);

}  // namespace he
