// he_kernels.h -- kernel declarations and their argument structs.
#pragma once
#include "he_common.cuh"

#define HE_MAX_DIGIT 8
#define HE_MAX_ROT 16  // rotations one hoisted rotate-and-sum stage may take

namespace he {

// A uniform batch of ciphertexts: ciphertext i, part p, limb t at
// base + i*stride + (p*cap + t)*N.
struct CtBatch {
  uint64_t* base;
  uint64_t stride;
  uint32_t cap;
  uint32_t pad;
};

// Ciphertext i, part p, limb t of a uniform batch.
__device__ __forceinline__ uint64_t* cpoly(const CtBatch& b, uint32_t i, uint32_t p, uint32_t t, uint32_t n) {
  return b.base + (size_t)i * b.stride + ((size_t)p * b.cap + t) * n;
}

struct ModUpArgs {
  uint32_t level, alpha, beta, L, np;
  uint32_t lo[HE_MAX_PRIMES], cnt[HE_MAX_PRIMES];
  uint64_t off[HE_MAX_PRIMES];
};

// The rotations of one hoisted rotate-and-sum: Galois elements and keys.
struct RotSet {
  uint32_t n;
  uint64_t gal[HE_MAX_ROT];
  const uint64_t* evk[HE_MAX_ROT];
};

struct LimbConsts {
  uint64_t w[HE_MAX_PRIMES];
  uint64_t wsh[HE_MAX_PRIMES];
};

__global__ void k_tensor(CtBatch A, CtBatch B, CtBatch D, uint64_t* d2, uint64_t d2_stride,
                         uint32_t level, uint32_t count, int log_n, const PrimeDev* primes);
__global__ void k_modup(const uint64_t* xc, uint64_t xc_stride, uint64_t* ext, uint64_t ext_stride,
                        ModUpArgs m, uint32_t count, int log_n, const PrimeDev* primes,
                        const uint64_t* consts);
__global__ void k_inner_product(const uint64_t* ext, uint64_t ext_stride, const uint64_t* d,
                                uint64_t d_stride, const uint64_t* evk, uint64_t* acc,
                                uint64_t acc_stride, uint32_t level, uint32_t alpha, uint32_t beta,
                                uint32_t L, uint32_t np, uint32_t count, int log_n,
                                const PrimeDev* primes);
__global__ void k_inner_product_rot(const uint64_t* ext, uint64_t ext_stride, const uint64_t* d,
                                    uint64_t d_stride, RotSet rs, uint64_t* acc, uint64_t acc_stride,
                                    uint32_t level, uint32_t alpha, uint32_t beta, uint32_t L, uint32_t np,
                                    uint32_t count, int log_n, const PrimeDev* primes);
__global__ void k_reduce_acc(uint64_t* acc, uint64_t acc_stride, uint32_t nt, uint32_t level, uint32_t L,
                             uint32_t count, int log_n, const PrimeDev* primes);
__global__ void k_add_automorphs(CtBatch A, CtBatch O, RotSet rs, uint32_t level, uint32_t count, int log_n,
                                 const PrimeDev* primes);
// The dropped limbs of a ModDown: n limbs of acc starting at limb `first`,
// over the primes pr[0 .. n).
struct MdDrop {
  uint32_t n, first;
  uint32_t pr[HE_MAX_DIGIT];
};
__global__ void k_moddown_conv(const uint64_t* acc, uint64_t acc_stride, uint32_t nt, MdDrop dr, uint64_t* conv,
                               uint64_t conv_stride, uint32_t level, uint32_t L, uint32_t count, int log_n,
                               const PrimeDev* primes, const uint64_t* md);
__global__ void k_ks_combine(const uint64_t* acc, uint64_t acc_stride, uint32_t nt, const uint64_t* conv,
                             uint64_t conv_stride, CtBatch add, int has_add, const uint64_t* addw, CtBatch out,
                             uint32_t level, uint32_t count, int log_n, const PrimeDev* primes,
                             const uint64_t* pinv);
__global__ void k_add_pd(uint64_t* acc, uint64_t acc_stride, uint32_t nt, CtBatch d, uint32_t l, uint64_t Pl,
                         uint64_t Pl_sh, uint32_t count, int log_n, const PrimeDev* primes);
__global__ void k_rescale_corr(const uint64_t* last, uint64_t* corr, uint32_t level, uint32_t count,
                               int log_n, const PrimeDev* primes);
__global__ void k_rescale_final(CtBatch in, const uint64_t* corr, CtBatch out, uint32_t level,
                                uint32_t count, int log_n, const PrimeDev* primes, const uint64_t* rs);
__global__ void k_automorph(CtBatch in, CtBatch out, uint32_t nparts, uint32_t level, uint64_t gal,
                            uint32_t count, int log_n);
__global__ void k_addsub(CtBatch A, CtBatch B, CtBatch O, int op, uint32_t level, uint32_t count,
                         int log_n, const PrimeDev* primes);
__global__ void k_mul_const(CtBatch A, CtBatch O, LimbConsts kc, uint32_t level, uint32_t count,
                            int log_n, const PrimeDev* primes);
__global__ void k_add_const(CtBatch A, CtBatch O, LimbConsts kc, uint32_t level, uint32_t count,
                            int log_n, const PrimeDev* primes);
__global__ void k_mul_plain(CtBatch A, const uint64_t* pt, CtBatch O, uint32_t level, uint32_t count,
                            int log_n, const PrimeDev* primes);
__global__ void k_copy_limbs(CtBatch A, CtBatch O, uint32_t level, uint32_t count, int log_n);

// keys.cu
__global__ void k_sample(uint64_t* out, uint64_t out_stride, uint32_t kind, uint32_t nl,
                         uint32_t limb0, uint32_t level, uint32_t L, uint64_t seed, uint32_t sid,
                         uint32_t dom, const uint64_t* gauss, int gK, uint32_t count, uint32_t sid_step,
                         int log_n, const PrimeDev* primes, const uint64_t* two64);
__global__ void k_signed_to_residues(const int64_t* src, uint64_t* out, uint32_t nl, int log_n,
                                     const PrimeDev* primes);

// codec.cu
__global__ void k_decrypt_dot(CtBatch A, const uint64_t* s, uint64_t* m, uint32_t level, int log_n,
                              const PrimeDev* primes);

}  // namespace he
