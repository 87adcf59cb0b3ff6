/*
 * he_gb300.h -- C ABI of the GB300 (sm_103a) library for the encrypted
 * logistic-regression worker step of Li & Huang, "Faster Secure Data Mining
 * via Distributed Homomorphic Encryption" (KDD'20).
 *
 * The paper's workers evaluate the linearised gradient update (Sec. 4,
 * Eq. 7-8, Table 2) on CKKS ciphertexts (Sec. 3: encode/decode,
 * encrypt/decrypt, addition, multiplication, rescaling) without
 * bootstrapping, and hand the encrypted weights back to the key holder for
 * a refresh every few iterations (Algorithm 1, Algorithm 2).  This library
 * implements that arithmetic in its full-RNS form: residues modulo word-size
 * primes q_0 > ... > q_{L-1} (the ciphertext modulus, "M" of Sec. 3) and
 * alpha special primes (the key-switching modulus P), ring degree N
 * ("N" of Sec. 3), N/2 complex slots.
 *
 * Conventions shared by every entry point
 *  - Ciphertext residues live in device memory (HBM) and are owned by the
 *    caller.  A ciphertext at level l (l limbs) in a buffer of `cap` limbs per
 *    part keeps part p (0 or 1), limb t (prime q_t) at
 *    data + (p*cap + t)*N, as N uint64 words in [0, q_t), in evaluation
 *    (NTT) form: word j is the value at psi_t^(2*brv(j)+1), psi_t the least
 *    primitive 2N-th root of unity mod q_t.  The buffer must hold 2*cap*N
 *    words, cap >= level.
 *  - Every call is asynchronous on the context's stream unless stated; host
 *    buffers passed in are read before the call returns; host results are
 *    complete when the call returns.
 *  - Every call returns HE_OK (0) or an error code below; a description of
 *    the last error on the calling thread is returned by he_last_error().
 *    Calls never modify their input ciphertexts; an output may alias an
 *    input only where stated.
 */
#ifndef HE_GB300_H
#define HE_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  HE_OK = 0,
  HE_EINVAL = 1,   /* null pointer, bad size, level or capacity */
  HE_ELEVEL = 2,   /* too few limbs left: the key holder must refresh (Alg. 1) */
  HE_ESCALE = 3,   /* operands' scales differ by more than 2^-40 relative */
  HE_ENOKEY = 4,   /* no Galois key for the requested rotation */
  HE_ENOMEM = 5,   /* device memory exhausted or budget exceeded */
  HE_ECUDA = 6,    /* CUDA runtime error */
  HE_ETIMEOUT = 7  /* a bounded device wait gave up */
};

/* Scheme parameters (Sec. 3 names two: the ring degree N and the modulus
 * size M; the rest are the RNS form's).  limb_bits/special_bits must be in
 * [20, 61]; scale is the default encoding scale Delta; sigma the standard
 * deviation of the discrete Gaussian errors; seed keys every random stream. */
typedef struct he_params {
  uint32_t log_n;        /* N = 2^log_n, 4 <= log_n <= 16 */
  uint32_t n_limbs;      /* L: limb primes q_0..q_{L-1} */
  uint32_t limb_bits;
  uint32_t n_special;    /* alpha: special primes (key-switching digit size), 1 .. 7 */
  uint32_t special_bits;
  uint32_t dnum;         /* 0, or must equal ceil(L / alpha) */
  double scale;
  double sigma;
  uint64_t seed;
} he_params;

typedef struct he_ctx he_ctx;

typedef struct he_ct {
  uint64_t* data;  /* device, 2*cap*N words */
  uint32_t level;  /* limbs in use */
  uint32_t cap;    /* limbs per part the buffer holds */
  double scale;    /* scale of the encoded message */
} he_ct;

/* Last error message of the calling thread ("" if none). */
const char* he_last_error(void);

/* Key generation from the seed (Algorithm 2, line 4: the parameter server
 * generates pk and sk).  Finds the primes (q = 1 mod 2N, scanned downward
 * from 2^bits), the secret s (ternary), the public key, the relinearisation
 * key and one Galois key per distinct rotation step in rot_steps[0..n_rot)
 * (steps are reduced mod N/2; 0 is ignored).  `stream` is a cudaStream_t (NULL
 * = the legacy default stream) on which every later call runs.  Keys stay
 * resident in device memory owned by the context.  Errors: HE_EINVAL,
 * HE_ENOMEM, HE_ECUDA. */
int he_ctx_create(const he_params* params, const int32_t* rot_steps, size_t n_rot, void* stream,
                  he_ctx** out);
int he_ctx_destroy(he_ctx* ctx);
/* Switch the stream later calls run on (cudaStream_t). */
int he_set_stream(he_ctx* ctx, void* stream);
/* Synchronise the context's stream. */
int he_sync(he_ctx* ctx);

/* Tuning knobs (results never depend on them): "chunk_bytes" = scratch budget
 * of one batched operation (default 2^34), "lr_chunk" = data ciphertexts per
 * chunk of the logistic-regression step (0 = from the budget), "ntt_generic"
 * = 1 to run the runtime-shaped NTT kernel instead of the compile-time-shaped
 * one for N = 2^12 .. 2^16, "ntt_shape" = 0 (default), 1 or 2 for the three NTT tile-shape pairs compiled
 * per ring size (also used by the fused key switch), "ntt_pb_max" = at most this
 * many polynomials of one limb per NTT CTA (default 8), "ks_ct" = 1, 2 or 4
 * ciphertexts per CTA of the key switch's product kernel in stages whose
 * rotations keep each CTA's rows (0, the default: 2 when their tiles fit in
 * shared memory).  HE_EINVAL for an unknown key or a value out of range. */
int he_set_tuning(he_ctx* ctx, const char* key, double value);
/* Current value of a tuning knob (the keys above). */
int he_get_tuning(he_ctx* ctx, const char* key, double* value);

/* Measurement utility (no counterpart in the paper): register-resident
 * throughput on the current device of kind 0 = 32-bit multiply-adds, 1 =
 * 64-bit Shoup modular products (the integer roof of the transforms), 2 =
 * radix-8 rounds of the lazy forward butterfly, 3 = 64 x 64 -> 128-bit
 * multiply-accumulates (the key switch's unreduced key products on wide
 * primes), 4 = split key products of residues below 2^40 (three 32 x 32 ->
 * 64-bit multiply-adds each, the key products on narrower primes); per clock
 * per SM (at the device's maximum clock) and per second.  Runs two short
 * kernels on the default stream and synchronises. */
int he_probe_alu(int kind, double* per_clock_per_sm, double* per_second);

/* Least-squares polynomial fit of a nonlinearity from samples (Sec. 3,
 * Eq. 3), the host utility behind gradient polynomials such as Table 2's:
 * coeffs[0..degree] minimise sum_i (y_i - sum_k coeffs[k] x_i^k)^2 over the n
 * samples (x_i, y_i).  Host memory, host computation (no device, no context);
 * degree <= 16, n > degree.  HE_EINVAL for null pointers, a non-finite sample,
 * too few samples or samples that do not determine the polynomial (fewer
 * than degree + 1 distinct abscissas).  Table 2's binomial row is the fit of
 * the negated logistic-loss derivative 1/(1+e^x) on [-16, 16] (evenly spaced
 * samples), to its printed digits. */
int he_fit_poly(const double* x, const double* y, size_t n, uint32_t degree, double* coeffs);

/* Autotuner (no counterpart in the paper; it serves the batched workers of
 * Sec. 4): times the relinearisation key switch (iNTT, ModUp + NTT, inner
 * product, ModDown) of `count` polynomials of uniform residues at `level`
 * under every setting of "ntt_shape" and "ntt_pb_max" in {1, 4, 8}, keeps the fastest in the context and writes its time per key
 * switch (ms) to *best_ms (may be NULL).  Synchronises the context's stream;
 * results never depend on these knobs.  HE_EINVAL for level outside [1, L] or
 * count outside [1, 4096]; on an error the knobs keep their previous values. */
int he_autotune(he_ctx* ctx, uint32_t level, uint32_t count, double* best_ms);

/* The context's workspace: the device bytes it holds now (scratch that the
 * entry points needing it grow on demand, key generation included) and how
 * many times an entry point has asked it for scratch, whether or not it grew.
 * Either output may be NULL. */
int he_ctx_workspace(const he_ctx* ctx, size_t* bytes, uint64_t* requests);

/* Context facts: N, L, alpha, beta (digits at the top level), and the
 * L + alpha primes (limbs first) into primes_out (may be NULL). */
int he_ctx_info(const he_ctx* ctx, uint32_t* n, uint32_t* n_limbs, uint32_t* n_special,
                uint32_t* beta, uint64_t* primes_out);

/* Encode (Sec. 3, canonical embedding): n_slots <= N/2 real values (host)
 * at `scale` into N integer coefficients (host), coefficient
 * i = round((2*scale/N) * sum_j Re(z_j * zeta_j^-i)), zeta_j = exp(i*pi*5^j/N),
 * rounding half away from zero; computed on the device in double
 * precision.  HE_EINVAL if a coefficient leaves int64. */
int he_encode(he_ctx* ctx, const double* slots, size_t n_slots, double scale, int64_t* coeffs_out);

/* Encrypt integer coefficients (host, N of them) at `level` (Sec. 3;
 * Algorithm 1 uses pk, Algorithm 2 encrypts with sk).
 * use_sk = 0: (v*b + e0 + m, v*a + e1); use_sk = 1: (-a*s + e + m, a).  The
 * randomness is the stream of ciphertext id `cid`, so equal inputs give
 * equal residues.  out->data must be allocated; sets level and scale. */
int he_encrypt_poly(he_ctx* ctx, const int64_t* coeffs, double scale, uint32_t level, int use_sk,
                    uint32_t cid, he_ct* out);

/* he_encode followed by he_encrypt_poly. */
int he_encode_encrypt(he_ctx* ctx, const double* slots, size_t n_slots, double scale,
                      uint32_t level, int use_sk, uint32_t cid, he_ct* out);

/* Decrypt to centered coefficients: m = c0 + c1*s mod Q_level, lifted to
 * (-Q/2, Q/2] and written as doubles (host, N values).  Synchronous. */
int he_decrypt_poly(he_ctx* ctx, const he_ct* ct, double* coeffs_out);

/* Decrypt and decode (Sec. 3): real parts of the first n_slots slots, each
 * divided by the ciphertext's scale (host).  Synchronous. */
int he_decrypt_decode(he_ctx* ctx, const he_ct* ct, double* slots_out, size_t n_slots);

/* Library-owned ciphertexts (the handle form of the conventions above): a
 * device buffer of 2*cap*N words allocated by the library (cap limbs per
 * part, 1 <= cap <= L), level 0 until an entry point writes it; pass the
 * handle wherever an he_ct* is taken.  he_ct_free synchronises the device
 * (work queued on any stream may still use the buffer), then frees the buffer
 * and the handle; NULL is ignored.  HE_EINVAL for a bad capacity, HE_ENOMEM
 * when device memory is exhausted.  Caller-owned buffers (an he_ct the caller
 * fills in) remain accepted everywhere. */
int he_ct_alloc(he_ctx* ctx, uint32_t cap, he_ct** out);
int he_ct_free(he_ct* ct);

/* Residues to and from host memory, packed [2][level][N] (uint64).  Export is
 * synchronous; cap_words is the capacity of `host` in words. */
int he_ct_export(he_ctx* ctx, const he_ct* ct, uint64_t* host, size_t cap_words);
int he_ct_import(he_ctx* ctx, const uint64_t* host, uint32_t level, double scale, he_ct* out);

/* Batched transfers of `count` ciphertexts packed [count][2][level][N] in
 * host memory (pinned memory gives full copy bandwidth).  Import sets every
 * out[i] to (level, scale); both are synchronous. */
int he_ct_import_batch(he_ctx* ctx, const uint64_t* host, uint32_t level, double scale, he_ct* out,
                       size_t count);
int he_ct_export_batch(he_ctx* ctx, const he_ct* cts, size_t count, uint64_t* host, size_t cap_words);

/* Homomorphic addition / subtraction (Sec. 3; Eq. 1-2).  Operands at
 * different levels are taken at the lower one.  HE_ESCALE if the scales
 * differ.  out may alias a or b. */
int he_add(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out);
int he_sub(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out);

/* out = a[0] + ... + a[count-1] (Eq. 1 applied count - 1 times): residues
 * added modulo each limb's prime, in one kernel when a[1..count) sit at a
 * constant stride in one allocation.  The sum is taken at the lowest level
 * of the inputs, all at one scale (else HE_ESCALE); out may alias a[0] only.
 * The aggregation of several workers' encrypted weights (Algorithm 2). */
int he_sum(he_ctx* ctx, const he_ct* a, size_t count, he_ct* out);

/* Keep the first `level` limbs (modulus reduction without division). */
int he_drop_level(he_ctx* ctx, const he_ct* a, uint32_t level, he_ct* out);

/* Multiply by the integer round(value * value_scale) (a constant plaintext
 * at scale value_scale); out.scale = a.scale * value_scale.  No rescale. */
int he_mul_const(he_ctx* ctx, const he_ct* a, double value, double value_scale, he_ct* out);

/* Add the constant `value` (encoded as round(value * a.scale)). */
int he_add_const(he_ctx* ctx, const he_ct* a, double value, he_ct* out);

/* Multiply by a plaintext given as N integer coefficients (host) at scale
 * pt_scale; out.scale = a.scale * pt_scale.  No rescale. */
int he_mul_plain(he_ctx* ctx, const he_ct* a, const int64_t* coeffs, double pt_scale, he_ct* out);

/* Rescale (Sec. 3 "scaling performs homomorphic rounding"): divide by the
 * last limb prime q_{l-1} with rounding, out at level l-1, scale / q_{l-1}.
 * HE_ELEVEL if l < 2. */
int he_rescale(he_ctx* ctx, const he_ct* a, he_ct* out);

/* he_rescale without any device allocation (the paper has no counterpart:
 * this is a deployment variant).  he_rescale draws its scratch from the
 * context's workspace, which may grow with cudaMalloc and synchronise the
 * stream; callers that cannot allow that (a host that owns the device's
 * memory through its own pool and a fixed HBM budget, or a latency-critical
 * loop that must not stall on an allocation) use this entry point, whose
 * scratch is a static 4 MiB device array present on every GPU that loads the
 * library until exit.  Limit: 2*level*N + 64 words <= 2^19 (level <= 15 at
 * N = 2^14), else HE_EINVAL with the sizes in the message.  The first call on
 * a device looks up the array's device address with that device current;
 * make that first call before any stream capture.  The address is kept for
 * the life of the process, which assumes the device's primary context is
 * never reset: after cudaDeviceReset do not call this entry point again.
 * The context's workspace (he_ctx_workspace) is neither used nor grown, and
 * kernel timing (he_profile_*) is skipped for this call.  All calls share the
 * array: calls that overlap on the GPU race, so serialise them; nothing in
 * it needs clearing, each call writes every word it reads.  Same results,
 * errors and aliasing rules as he_rescale; kernel timing is not recorded. */
int he_rescale_noalloc(he_ctx* ctx, const he_ct* a, he_ct* out);

/* Homomorphic multiplication (Sec. 3; the cost the paper names in Sec. 6):
 * tensor product (d0, d1, d2), relinearisation by hybrid key switching, and
 * rescale, the key switch's division by P and the rescale's by q_{l-1} taken
 * as one rounding: out = round((P (d0, d1) + <ModUp(d2), rlk>) / (P q_{l-1})).
 * Both operands at the same level l >= 2 (else the lower is used); out at
 * l-1 with scale a.scale*b.scale/q_{l-1}. */
int he_mul_relin_rescale(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out);

/* Same, without the rescale (out at level l, scale a.scale*b.scale). */
int he_mul_relin(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out);

/* Rotate the slots left by `steps` (slot j <- slot j + steps), the packing
 * primitive behind the sums of Sec. 3-4: Galois automorphism X -> X^(5^steps)
 * and key switching.  HE_ENOKEY if the context has no key for the step. */
int he_rotate(he_ctx* ctx, const he_ct* a, int32_t steps, he_ct* out);

/* Batched forms: count independent operations in one launch sequence.  All
 * inputs of one call share level and scale. */
int he_mul_relin_rescale_batch(he_ctx* ctx, const he_ct* a, const he_ct* b, he_ct* out,
                               size_t count);
int he_rotate_batch(he_ctx* ctx, const he_ct* a, int32_t steps, he_ct* out, size_t count);

/* Rotate-and-sum with one shared decomposition: out = a + sum_{r < nsteps}
 * rotate(a, steps[r]), 1 <= nsteps <= 16, the sums over slot positions that
 * the packing of Sec. 3-4 reads inner products from.  The key switches of all
 * nsteps rotations share the ModUp of a's second part (each rotation applies
 * its automorphism to the raised digits) and one ModDown of their summed
 * inner products, so a stage of three rotations costs about one and a half
 * key switches instead of three.  Its residues differ from those of
 * he_rotate + he_add (the approximate basis conversion does not commute with
 * the automorphism's sign flips) but it decrypts to the same sum with the
 * noise of one key switch.  out (level and scale of a) may be a; other
 * overlaps of inputs and outputs are refused (HE_EINVAL).  HE_ENOKEY if a
 * step has no Galois key, HE_EINVAL for a step of 0 slots.  The batched form
 * takes count ciphertexts of one level. */
int he_rotate_sum(he_ctx* ctx, const he_ct* a, const int32_t* steps, uint32_t nsteps, he_ct* out);
int he_rotate_sum_batch(he_ctx* ctx, const he_ct* a, const int32_t* steps, uint32_t nsteps, he_ct* out,
                        size_t count);

/* Encrypted logistic-regression gradient step (Sec. 4: Eq. 5-8 with a Table 2
 * polynomial; Algorithm 1).  Z[k] hold g samples each, slot g*f + s =
 * y_s*x_{s,f}; W holds w_f in slots g*f + s for every s.  Computes
 * w' = w + lr * sum_k sum_s p(y_s w.x_s) y_s x_s with p(x) = c0 + c1 x +
 * c2 x^2 + c3 x^3, replicated over the g slots of each feature (minus
 * lr * l2 * w with the L2 regulariser below).  Consumes 5
 * levels: Z and W at the same level l >= 6; W_out at l - 5 with W's scale.
 * Each of its three rotate-and-sums (over F = N/(2g) feature positions of
 * step g, and over the g samples with steps 1 and -1) runs as he_rotate_sum
 * stages of k doublings each -- steps s, 2s, ..., (2^k - 1)s, then s <- 2^k s
 * -- with k = 3, except k = 4 for the first stage when the number of
 * doublings is 1 mod 3 (k = 1 if it is 1) and k = 2 for a last stage when it
 * is 2 mod 3.  Needs Galois keys for all those steps (lr_rot_steps in the
 * Python binding lists them; e.g. g = 8, F = 1024: 8, 16, ..., 120, then
 * 128, ..., 896, then 1024, ..., 7168, and 1, ..., 7 and -1, ..., -7). */
typedef struct he_lr_config {
  double coeffs[4];     /* c0..c3 */
  double lr;            /* learning rate, e.g. eta / n */
  uint32_t g;           /* samples per ciphertext, a power of two */
  uint32_t pad;
  double mask_scale;    /* scale of the 0/1 slot mask plaintext */
  double l2;            /* >= 0: weight of the regulariser R(w) = (l2/2) |w|^2 of Eq. 4, whose
                           gradient l2 w joins the sum (Eq. 6, 8): w' = w + lr (sum ... - l2 w);
                           taken as round(-lr l2 q_{l-6}) times w at level l - 4, rescaled to
                           l - 5 and W's scale, and added last (0: no regulariser) */
} he_lr_config;

int he_lr_gradient_step(he_ctx* ctx, const he_ct* Z, size_t nZ, const he_ct* W,
                        const he_lr_config* cfg, he_ct* W_out);

/* The same step (Eq. 7-8) with its inputs and result in host memory, the way
 * a worker receives its encrypted shard (Algorithm 1): Z = nZ ciphertexts of
 * [2][z_level][N] residues back to back, W = [2][w_level][N] (6 <= w_level <=
 * z_level <= L); the result [2][w_level-5][N] goes to `out` (out_words >= its
 * size), its level and scale to *out_level / *out_scale (may be NULL).  The
 * weights and then pieces of 16 data ciphertexts are copied on a second
 * stream while the circuit runs chunk by chunk on the context's stream, so
 * the copies overlap the arithmetic (unless lr_chunk is set, a short first
 * chunk, sized from the copy and arithmetic times of the previous call, then
 * chunks of the scratch budget); pinned host memory is needed for that
 * overlap (pageable memory is copied synchronously).  Returns after the
 * result is in `out`.  The device copy of the inputs is a context-owned
 * buffer, grown on demand.  HE_ELEVEL if w_level < 6. */
int he_lr_gradient_step_host(he_ctx* ctx, const uint64_t* Z, size_t nZ, uint32_t z_level, double z_scale,
                             const uint64_t* W, uint32_t w_level, double w_scale, const he_lr_config* cfg,
                             uint64_t* out, size_t out_words, uint32_t* out_level, double* out_scale);

/* The paper's K workers (Sec. 4, Fig. 1; Algorithm 1) as independent
 * instances on one GPU, all stepped in one batched launch sequence.  Shard k
 * holds its own data ciphertexts Z[0..nZ) (one level, one scale), its weights
 * W and an output buffer W_out.  A shard whose weights sit below level 6 (too
 * few limbs for the step's five rescales) first goes through the in-process
 * key-holder refresh (Algorithm 1) to refresh_level (0 = refuse
 * with HE_ELEVEL); the step then runs at the weights' level l with the data
 * taken at l, and W_out receives level l - 5 and W's scale.  Shards with the
 * same level and scales share every kernel launch; their data ciphertexts
 * are processed together in chunks.  With HE_LR_GRAPH the whole launch
 * sequence is captured once per distinct call (same buffers, sizes and
 * configuration) as a CUDA graph and replayed; this needs a non-default
 * stream, and a replay reuses the refresh encryptions' random streams. */
typedef struct he_lr_shard {
  const he_ct* Z;        /* nZ data ciphertexts */
  size_t nZ;
  const he_ct* W;        /* encrypted weights */
  he_ct* W_out;          /* gradient step: the new weights */
  he_ct* S_out;          /* inference: nZ outputs, S_k = p(M_k) (may be NULL for the step) */
  uint32_t refresh_cid;  /* ciphertext id of the refresh encryption (if one is needed) */
  uint32_t min_level;    /* refresh the weights first when their level is below this;
                            0 (or less than the circuit needs) = the circuit's minimum:
                            6 for the step, 5 for inference */
} he_lr_shard;

#define HE_LR_GRAPH 1

int he_lr_gradient_step_workers(he_ctx* ctx, const he_lr_shard* shards, size_t count,
                                const he_lr_config* cfg, uint32_t refresh_level, int flags);

/* The training loop of Algorithms 1 and 2 in one process: worker k (shard
 * k: data Z[0..nZ), initial weights W at top_level, all at one scale; W_out
 * and S_out unused) runs `iterations` gradient steps (Eq. 7-8, this cfg) on
 * its own data from its own weights; after every `refresh_every` steps and
 * after the last, the key holder (Algorithm 2) decrypts all
 * workers' weights, averages them slot by slot (the paper leaves its update
 * rule open), encodes the average at the weights' scale and encrypts it once
 * at top_level (random stream cid0 + iteration), and every worker continues
 * from that ciphertext.  W_final (cap >= top_level) receives the last
 * average.  Needs top_level >= 5 * refresh_every + 1 (a step consumes 5
 * limbs), else HE_ELEVEL; HE_EINVAL for weights not at top_level; HE_ESCALE
 * for different scales.  Weight buffers are allocated for the call. */
int he_lr_train(he_ctx* ctx, const he_lr_shard* shards, size_t count, const he_lr_config* cfg,
                uint32_t iterations, uint32_t refresh_every, uint32_t top_level, uint32_t cid0, he_ct* W_final);

/* Encrypted inference of the same model (the first half of the step): for
 * every data ciphertext Z_k of every shard, S_k = p(M_k) with M_k = the
 * per-sample inner products y_s w.x_s replicated over each sample's slots
 * (packing as in he_lr_gradient_step) and p the configured cubic (c_i * lr).
 * S_out[k] receives level l - 3 and W's scale (l = the weights' level after
 * any refresh, which must be >= 5 so that the result keeps two limbs).
 * Grouping, refresh and graph capture as in he_lr_gradient_step_workers. */
int he_lr_inference_workers(he_ctx* ctx, const he_lr_shard* shards, size_t count,
                            const he_lr_config* cfg, uint32_t refresh_level, int flags);

/* ---- Serving: a continuous-batching request loop ----------------------------
 * The paper's workers answer gradient steps (Algorithm 1) and, with
 * the same model, inference.  A server holds contexts of several ring sizes
 * (keys resident in HBM) and a scheduler thread.  Requests carry host
 * residues; the scheduler admits them oldest first while their device memory
 * (inputs, outputs) plus the slots' workspaces stay within hbm_budget, groups
 * pending requests with the same context, kind, data level, scales and
 * configuration into a wave of at most max_wave, and runs each wave as one
 * batched call on one of max_inflight streams per context: requests arriving
 * while waves run join the next free slot without waiting for the others, and
 * waves on different streams overlap on the device.  A request whose weights
 * have too few limbs is refreshed in-process to the data's level first, with
 * random stream refresh_cid, so its result does not depend on its wave.
 * Calls return HE_OK or an error code: HE_EINVAL for null or inconsistent
 * arguments (context index, kind, levels, output size), HE_ELEVEL at submit
 * for data below the circuit's depth, HE_ETIMEOUT from drain; a failure while
 * running a wave (HE_ENOMEM, HE_ECUDA, ...) is reported in the status of each
 * of its requests' results.  The server owns its streams, slot views and
 * scheduler thread; destroy joins the thread after the queued work. */
enum { HE_REQ_GRADIENT = 0, HE_REQ_INFERENCE = 1 };

typedef struct he_server he_server;

typedef struct he_server_config {
  he_ctx* const* ctxs;    /* contexts, one per ring size class; not owned */
  size_t n_ctx;
  size_t hbm_budget;      /* bytes of device memory for request buffers and workspaces */
  uint32_t max_inflight;  /* concurrent waves per context (streams), 1..16 */
  uint32_t max_wave;      /* requests per wave */
  uint32_t max_running;   /* waves in flight over all contexts; 0 = no limit beyond
                             max_inflight per context (1 with max_wave 1 serves one
                             request at a time) */
} he_server_config;

typedef struct he_request {
  uint32_t ctx;          /* index into the server's contexts */
  uint32_t kind;         /* HE_REQ_GRADIENT or HE_REQ_INFERENCE */
  uint32_t nZ;           /* data ciphertexts */
  uint32_t z_level;      /* level of the data (>= 6 for a step, >= 5 for inference) */
  uint32_t w_level;      /* level of the weights (<= z_level) */
  uint32_t refresh_cid;  /* ciphertext id of the refresh encryption, if one is needed */
  uint32_t min_w_level;  /* as he_lr_shard.min_level: e.g. 7 keeps a step's result at
                            two limbs or more */
  double z_scale, w_scale;
  const uint64_t* Z;     /* host, nZ x [2][z_level][N] residues (pinned memory keeps the loop asynchronous) */
  const uint64_t* W;     /* host, [2][w_level][N] */
  he_lr_config cfg;
  uint64_t* out;         /* host result: step [2][l-5][N], inference nZ x [2][l-3][N], l = weights' level
                            after any refresh (z_level when refreshed); pinned */
  size_t out_words;      /* capacity of out */
} he_request;

typedef struct he_result {
  uint64_t id;
  int32_t status;        /* HE_OK or the error of the request's wave */
  uint32_t level;        /* level of the result ciphertext(s) */
  double scale;          /* their scale */
  double latency_ms;     /* submit to completion seen by the scheduler */
} he_result;

int he_server_create(const he_server_config* cfg, he_server** out);
/* Queue a request (the descriptor is copied; host buffers must stay valid
 * until its result is polled).  Returns its id.  HE_ENOMEM (nothing queued)
 * for a request whose own device memory -- its buffers and the workspace of
 * its circuit -- exceeds the whole budget: it could never be admitted. */
int he_server_submit(he_server* s, const he_request* req, uint64_t* id);
/* Results completed since the last poll (up to cap). */
int he_server_poll(he_server* s, he_result* results, size_t cap, size_t* n);
/* Wait until nothing is pending or running (HE_ETIMEOUT after timeout_s). */
int he_server_drain(he_server* s, double timeout_s);
/* Device bytes held now and at most so far (request buffers and slot
 * workspaces), waves launched, and the most waves running at once. */
int he_server_stats(he_server* s, size_t* used, size_t* peak_used, size_t* waves, size_t* peak_running);
/* The message of the most recent failed wave (empty if none), copied to buf
 * (cap bytes including the terminating zero). */
int he_server_last_error(he_server* s, char* buf, size_t cap);
int he_server_destroy(he_server* s);

/* The key holder's refresh (Algorithm 1, Algorithm 2),
 * simulated in-process: decrypt, decode, re-encode at out_scale and encrypt
 * at `level` with ciphertext id cid.  Synchronous. */
int he_refresh(he_ctx* ctx, const he_ct* a, uint32_t level, double out_scale, uint32_t cid,
               he_ct* out);

/* Low-level entry points for kernel parity tests. */
/* Forward (inverse = 0) or inverse negacyclic NTT of `nl` limbs (limb t with
 * prime index prime0 + t) of `npolys` device polynomials at data +
 * p*poly_stride words, in place. */
int he_ntt(he_ctx* ctx, uint64_t* data, uint32_t npolys, uint64_t poly_stride, uint32_t nl,
           uint32_t prime0, int inverse);
/* Hybrid key switching of d (device, level limbs, evaluation form) with the
 * relinearisation key (galois = 0) or the Galois key of element `galois`:
 * out0 + out1*s ~ d*s'.  out0/out1: device, level limbs each. */
int he_keyswitch(he_ctx* ctx, const uint64_t* d, uint32_t level, uint64_t galois, uint64_t* out0,
                 uint64_t* out1);
/* The key switch's last step alone (the ModDown of hybrid key switching
 * behind Sec. 3's multiplication and rotation), on accumulators the caller
 * chooses: acc (device, [2][level + alpha][N] evaluation form, limbs q_0 ..
 * q_{level-1} then the special primes p_0 .. p_{alpha-1}; not modified).
 * d01 == NULL: out = round(acc / P) at `level` (the exact lift of acc's
 * P-part, so every coefficient is rounded, whatever that lift is).
 * d01 != NULL (a ciphertext at `level` >= 2): out = round((P d01 + acc) /
 * (P q_{level-1})) at level - 1 with d01's scale, the multiplication's
 * merged ModDown and rescale.  out must not overlap d01.  HE_EINVAL for a
 * null or misaligned pointer or a bad level. */
int he_moddown(he_ctx* ctx, const uint64_t* acc, uint32_t level, const he_ct* d01, he_ct* out);

/* Kernel timing for measurement (not part of the paper's method).  While
 * enabled, every launch of an instrumented kernel class ("ntt", "intt",
 * "modup", "inner_product", "moddown_conv", "ks_combine", "rescale",
 * "tensor", "automorph", "elementwise") is bracketed by CUDA events on the
 * context's stream and its algorithmic work (butterflies for the
 * transforms, modular products otherwise) and algorithmic DRAM bytes are
 * added to the class.  Enabling or disabling resets the counters;
 * he_profile_read synchronises and returns launches, total device time (ms),
 * work and bytes of one class; he_profile_names lists the classes seen,
 * comma-separated, into buf (HE_EINVAL if cap is too small). */
int he_profile_enable(he_ctx* ctx, int enable);
int he_profile_read(he_ctx* ctx, const char* kernel_class, uint64_t* launches, double* total_ms,
                    double* work, double* bytes);
int he_profile_names(he_ctx* ctx, char* buf, size_t cap);
/* How a class's work (as counted by he_profile_read) splits by kind: NTT
 * butterflies; 64 x 64 -> 128-bit multiply-accumulates summed without
 * reduction (the key products of the fused key switch on wide primes); and
 * split key products, each three 32 x 32 -> 64-bit multiply-adds into 64-bit
 * sums (the key products on primes of up to about 50 bits); the rest is
 * Shoup or Barrett products (basis conversion, scaling, reductions).  Lets a
 * roofline weigh each kind at its own measured rate (he_probe_alu kinds 2,
 * 3, 4, 1).  Any output may be NULL. */
int he_profile_read_kinds(he_ctx* ctx, const char* kernel_class, double* butterflies, double* macs,
                          double* split_macs);

#ifdef __cplusplus
}
#endif

#endif /* HE_GB300_H */
