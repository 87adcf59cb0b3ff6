/*
 * he_oracle.c -- CPU oracle for the leveled RNS-CKKS ciphertext arithmetic of
 * the encrypted logistic-regression worker step of Li & Huang, "Faster Secure
 * Data Mining via Distributed Homomorphic Encryption" (KDD'20).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library may load, link or
 * call this file; only the tests, the smoke check and the benchmark's CPU
 * baseline leg do.  It shares no code, header, table or constant generator
 * with the CUDA library: every prime, root, table and formula below is
 * computed here from its definition.
 *
 * Style: plain and slow.  Every residue operation is exact (unsigned __int128
 * products reduced with '%'); transforms are the textbook definitions (O(N^2))
 * or the textbook radix-2 Cooley-Tukey / Gentleman-Sande loops (pinned against
 * the definition by the tests); CRT is done with an explicit little bignum.
 *
 * The paper (Sec. 3) delegates the scheme to HEAAN (Cheon-Kim-Kim-Song 2017,
 * "approximate numbers"); it states no parameters and no formulas for the
 * ring arithmetic.  Where it is silent this oracle follows the standard full
 * RNS variant of that scheme (Cheon-Han-Kim-Kim-Song 2018) with hybrid key
 * switching (Han-Ki 2020).  Every such reading is marked [ext] and every
 * free convention (prime order, root choice, random streams, samplers) is
 * spelled out where it is implemented.
 *
 * Threads: when built with OpenMP, independent limbs (key generation, the
 * key switch's targets, ModDown's targets) and, in the gradient step,
 * independent data ciphertexts run in parallel.  Every parallel loop writes
 * disjoint outputs, and the one shared sum (the step's gradient over the data
 * ciphertexts) is exact modular addition, so results do not depend on the
 * thread count.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
typedef __int128 i128;

/* Threads of the parallel loops (1 without OpenMP). */
void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_get_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

#define ORC_MAX_PRIMES 64

/* ------------------------------------------------------------------------ */
/* Exact modular arithmetic                                                  */
/* ------------------------------------------------------------------------ */

static uint64_t mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a * b) % q); }
static uint64_t addmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + b) % q); }
static uint64_t submod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)(((u128)a + q - (b % q)) % q); }

static uint64_t powmod(uint64_t a, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  a %= q;
  while (e) {
    if (e & 1) r = mulmod(r, a, q);
    a = mulmod(a, a, q);
    e >>= 1;
  }
  return r;
}

/* q prime: inverse by Fermat's little theorem. */
static uint64_t invmod(uint64_t a, uint64_t q) { return powmod(a % q, q - 2, q); }

/* Signed integer -> residue in [0, q). */
static uint64_t smod(int64_t x, uint64_t q) {
  i128 r = (i128)x % (i128)q;
  if (r < 0) r += q;
  return (uint64_t)r;
}

/* ------------------------------------------------------------------------ */
/* Primes and roots [ext]: q = 1 (mod 2N) so that X^N + 1 splits mod q.     */
/* ------------------------------------------------------------------------ */

/* Deterministic Miller-Rabin: the first twelve primes as bases decide every
 * n < 3.3e24, hence every 64-bit n. */
int orc_is_prime(uint64_t n) {
  static const uint64_t bases[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return 0;
  for (int i = 0; i < 12; i++) {
    if (n == bases[i]) return 1;
    if (n % bases[i] == 0) return 0;
  }
  uint64_t d = n - 1;
  int s = 0;
  while ((d & 1) == 0) { d >>= 1; s++; }
  for (int i = 0; i < 12; i++) {
    uint64_t x = powmod(bases[i], d, n);
    if (x == 1 || x == n - 1) continue;
    int comp = 1;
    for (int r = 1; r < s; r++) {
      x = mulmod(x, x, n);
      if (x == n - 1) { comp = 0; break; }
    }
    if (comp) return 0;
  }
  return 1;
}

/* Convention: scan q = k*2N + 1 downward from the largest such q below 2^bits
 * and keep the primes not listed in `exclude`, in the order found (so the
 * returned primes are strictly decreasing).  Returns the number found. */
int orc_gen_primes(int bits, int log_n, int count, const uint64_t* exclude, int n_ex,
                   uint64_t* out) {
  uint64_t two_n = (uint64_t)2 << log_n;
  uint64_t top = (bits >= 64) ? UINT64_MAX : (((uint64_t)1 << bits) - 1);
  uint64_t k = (top - 1) / two_n; /* largest k with k*2N + 1 <= 2^bits - 1 */
  int found = 0;
  while (found < count && k > 0) {
    uint64_t q = k * two_n + 1;
    int skip = 0;
    for (int i = 0; i < n_ex; i++)
      if (exclude[i] == q) skip = 1;
    if (!skip && orc_is_prime(q)) out[found++] = q;
    k--;
  }
  return found;
}

/* Convention: psi = the smallest residue of multiplicative order exactly 2N,
 * i.e. the least root of X^N + 1 mod q.  Found by taking a quadratic
 * non-residue g (the least one), psi0 = g^((q-1)/2N) (a primitive 2N-th
 * root), and the minimum over all odd powers psi0^(2k+1), which are exactly
 * the primitive 2N-th roots. */
uint64_t orc_min_root(uint64_t q, int log_n) {
  uint64_t n = (uint64_t)1 << log_n;
  uint64_t g = 2;
  while (powmod(g, (q - 1) / 2, q) != q - 1) g++;
  uint64_t psi0 = powmod(g, (q - 1) / (2 * n), q);
  uint64_t sq = mulmod(psi0, psi0, q);
  uint64_t cur = psi0, best = psi0;
  for (uint64_t k = 1; k < n; k++) {
    cur = mulmod(cur, sq, q);
    if (cur < best) best = cur;
  }
  return best;
}

/* ------------------------------------------------------------------------ */
/* Negacyclic NTT [ext].  Convention: evaluation at the odd powers of psi in  */
/* bit-reversed order:  A[j] = sum_i a[i] * psi^(i * (2*brv(j) + 1)) mod q.   */
/* ------------------------------------------------------------------------ */

static uint32_t brv(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; i++) { r = (r << 1) | (x & 1); x >>= 1; }
  return r;
}

/* The definition, O(N^2). */
void orc_ntt_def(const uint64_t* a, uint64_t* out, int log_n, uint64_t q, uint64_t psi) {
  uint32_t n = 1u << log_n;
  for (uint32_t j = 0; j < n; j++) {
    uint64_t e = 2 * (uint64_t)brv(j, log_n) + 1;
    uint64_t w = powmod(psi, e, q); /* psi^(2brv(j)+1) */
    uint64_t acc = 0, wp = 1;
    for (uint32_t i = 0; i < n; i++) {
      acc = addmod(acc, mulmod(a[i] % q, wp, q), q);
      wp = mulmod(wp, w, q);
    }
    out[j] = acc;
  }
}

/* The exact inverse of the definition, O(N^2):
 * a[i] = N^-1 * sum_j A[j] * psi^(-i * (2*brv(j) + 1)). */
void orc_intt_def(const uint64_t* A, uint64_t* out, int log_n, uint64_t q, uint64_t psi) {
  uint32_t n = 1u << log_n;
  uint64_t psi_inv = invmod(psi, q), n_inv = invmod(n, q);
  for (uint32_t i = 0; i < n; i++) {
    uint64_t acc = 0;
    for (uint32_t j = 0; j < n; j++) {
      uint64_t e = ((2 * (uint64_t)brv(j, log_n) + 1) * i) % (2 * (uint64_t)n);
      acc = addmod(acc, mulmod(A[j] % q, powmod(psi_inv, e, q), q), q);
    }
    out[i] = mulmod(acc, n_inv, q);
  }
}

/* Textbook in-place radix-2 negacyclic Cooley-Tukey (natural order in,
 * bit-reversed order out) with the table tw[m] = psi^brv(m). */
static void ntt_r2(uint64_t* a, int log_n, uint64_t q, const uint64_t* tw) {
  uint32_t n = 1u << log_n, t = n;
  for (uint32_t m = 1; m < n; m <<= 1) {
    t >>= 1;
    for (uint32_t i = 0; i < m; i++) {
      uint64_t w = tw[m + i];
      for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
        uint64_t u = a[j], v = mulmod(a[j + t], w, q);
        a[j] = addmod(u, v, q);
        a[j + t] = submod(u, v, q);
      }
    }
  }
}

/* Textbook in-place radix-2 Gentleman-Sande inverse (bit-reversed in,
 * natural out) with itw[m] = psi^-brv(m), then the factor N^-1. */
static void intt_r2(uint64_t* a, int log_n, uint64_t q, const uint64_t* itw, uint64_t n_inv) {
  uint32_t n = 1u << log_n, t = 1;
  for (uint32_t m = n; m > 1; m >>= 1) {
    uint32_t h = m >> 1;
    for (uint32_t i = 0; i < h; i++) {
      uint64_t w = itw[h + i];
      for (uint32_t j = 2 * i * t; j < 2 * i * t + t; j++) {
        uint64_t u = a[j], v = a[j + t];
        a[j] = addmod(u, v, q);
        a[j + t] = mulmod(submod(u, v, q), w, q);
      }
    }
    t <<= 1;
  }
  for (uint32_t i = 0; i < n; i++) a[i] = mulmod(a[i], n_inv, q);
}

static void make_tables(int log_n, uint64_t q, uint64_t psi, uint64_t* tw, uint64_t* itw) {
  uint32_t n = 1u << log_n;
  uint64_t psi_inv = invmod(psi, q);
  for (uint32_t m = 0; m < n; m++) {
    tw[m] = powmod(psi, brv(m, log_n), q);
    itw[m] = powmod(psi_inv, brv(m, log_n), q);
  }
}

/* Stand-alone radix-2 transforms (for pinning against the definition). */
void orc_ntt_r2(uint64_t* a, int log_n, uint64_t q, uint64_t psi) {
  uint32_t n = 1u << log_n;
  uint64_t* tw = malloc(sizeof(uint64_t) * n);
  uint64_t* itw = malloc(sizeof(uint64_t) * n);
  make_tables(log_n, q, psi, tw, itw);
  for (uint32_t i = 0; i < n; i++) a[i] %= q;
  ntt_r2(a, log_n, q, tw);
  free(tw);
  free(itw);
}

void orc_intt_r2(uint64_t* a, int log_n, uint64_t q, uint64_t psi) {
  uint32_t n = 1u << log_n;
  uint64_t* tw = malloc(sizeof(uint64_t) * n);
  uint64_t* itw = malloc(sizeof(uint64_t) * n);
  make_tables(log_n, q, psi, tw, itw);
  intt_r2(a, log_n, q, itw, invmod(n, q));
  free(tw);
  free(itw);
}

/* ------------------------------------------------------------------------ */
/* Randomness.  Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11), written   */
/* from its published definition: two multiply-xor S-boxes per round, Weyl   */
/* key schedule, ten rounds.                                                 */
/* ------------------------------------------------------------------------ */

void orc_philox(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; r++) {
    if (r > 0) { k0 += 0x9E3779B9u; k1 += 0xBB67AE85u; }
    uint64_t p0 = (uint64_t)0xD2511F53u * c0;
    uint64_t p1 = (uint64_t)0xCD9E8D57u * c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Stream convention: counter = (coefficient index, limb index or 0, stream
 * id, domain), key = (seed low word, seed high word). */
enum {
  DOM_S = 1, DOM_PK_A = 2, DOM_PK_E = 3, DOM_EVK_A = 4, DOM_EVK_E = 5,
  DOM_ENC_V = 6, DOM_ENC_E0 = 7, DOM_ENC_E1 = 8, DOM_ENC_A = 9
};

static void draw(uint64_t seed, uint32_t idx, uint32_t limb, uint32_t sid, uint32_t dom,
                 uint32_t out[4]) {
  uint32_t ctr[4] = {idx, limb, sid, dom};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox(ctr, key, out);
}

/* Ternary sampler: floor(3 * w0 / 2^32) - 1, uniform on {-1, 0, 1} up to
 * 2^-32 bias. */
static int sample_ternary(uint64_t seed, uint32_t idx, uint32_t sid, uint32_t dom) {
  uint32_t w[4];
  draw(seed, idx, 0, sid, dom, w);
  return (int)((((uint64_t)w[0]) * 3) >> 32) - 1;
}

/* Discrete Gaussian by cumulative table: K = ceil(6 sigma); rho_k =
 * exp(-k^2 / (2 sigma^2)); Z = rho_0 + 2 sum_{k=1..K} rho_k;
 * T[k] = floor(2^64 * (rho_0 + 2 sum_{i=1..k} rho_i) / Z) for k < K.
 * A draw u (64 bits) gives |x| = #{k < K : u >= T[k]}, sign from one bit. */
int orc_gauss_table(double sigma, uint64_t* T) {
  int K = (int)ceil(6.0 * sigma);
  double denom = 2.0 * sigma * sigma;
  double rho[256];
  if (K < 1 || K > 255) return -1;
  for (int k = 0; k <= K; k++) rho[k] = exp(-((double)(k * k)) / denom);
  double z = rho[0];
  for (int k = 1; k <= K; k++) z += 2.0 * rho[k];
  double cum = rho[0];
  T[0] = (uint64_t)ldexp(cum / z, 64);
  for (int k = 1; k < K; k++) {
    cum += 2.0 * rho[k];
    T[k] = (uint64_t)ldexp(cum / z, 64);
  }
  return K;
}

static int sample_gauss(uint64_t seed, uint32_t idx, uint32_t sid, uint32_t dom,
                        const uint64_t* T, int K) {
  uint32_t w[4];
  draw(seed, idx, 0, sid, dom, w);
  uint64_t u = ((uint64_t)w[1] << 32) | w[0];
  int k = 0;
  while (k < K && u >= T[k]) k++;
  return (w[2] & 1) ? -k : k;
}

/* Uniform residue: the 128-bit word (w3:w2:w1:w0) reduced mod q. */
static uint64_t sample_uniform(uint64_t seed, uint32_t idx, uint32_t limb, uint32_t sid,
                               uint32_t dom, uint64_t q) {
  uint32_t w[4];
  draw(seed, idx, limb, sid, dom, w);
  u128 x = ((u128)w[3] << 96) | ((u128)w[2] << 64) | ((u128)w[1] << 32) | (u128)w[0];
  return (uint64_t)(x % q);
}

/* Exposed for the sampler tests. */
void orc_sample(uint64_t seed, uint32_t kind, uint32_t sid, uint32_t dom, uint32_t limb,
                uint64_t q, double sigma, uint32_t count, int64_t* out) {
  uint64_t T[256];
  int K = orc_gauss_table(sigma, T);
  for (uint32_t i = 0; i < count; i++) {
    if (kind == 0) out[i] = sample_ternary(seed, i, sid, dom);
    else if (kind == 1) out[i] = sample_gauss(seed, i, sid, dom, T, K);
    else out[i] = (int64_t)sample_uniform(seed, i, limb, sid, dom, q);
  }
}

/* ------------------------------------------------------------------------ */
/* Context: parameters, keys.                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
  int32_t step;   /* rotation step r (slot j <- slot j + r) */
  uint64_t gal;   /* Galois element k = 5^r mod 2N */
  uint64_t* key;  /* [beta][2][L + alpha][N], evaluation form */
} orc_galkey;

typedef struct orc_ctx {
  int log_n, n, L, alpha, beta, np;
  double scale, sigma;
  uint64_t seed;
  uint64_t q[ORC_MAX_PRIMES];      /* q[0..L-1] limbs (decreasing), q[L..L+alpha-1] special */
  uint64_t psi[ORC_MAX_PRIMES];
  uint64_t* tw[ORC_MAX_PRIMES];
  uint64_t* itw[ORC_MAX_PRIMES];
  uint64_t ninv[ORC_MAX_PRIMES];
  uint64_t gT[256];
  int gK;
  int8_t* s_coef;                  /* [N] ternary secret */
  uint64_t* s;                     /* [np][N] evaluation form */
  uint64_t* pk_b;                  /* [L][N] */
  uint64_t* pk_a;                  /* [L][N] */
  uint64_t* rlk;                   /* [beta][2][np][N], s' = s^2 */
  int ngal;
  orc_galkey* gal;
  double* cos_t;                   /* cos(pi t / N), t in [0, 2N) */
  double* sin_t;
} orc_ctx;

#define POLY(base, idx, n) ((base) + (size_t)(idx) * (size_t)(n))

static void ntt_limb(orc_ctx* c, int t, uint64_t* a) { ntt_r2(a, c->log_n, c->q[t], c->tw[t]); }
static void intt_limb(orc_ctx* c, int t, uint64_t* a) { intt_r2(a, c->log_n, c->q[t], c->itw[t], c->ninv[t]); }

/* Digit D_j = limbs [j*alpha, min((j+1)*alpha, level)) (hybrid key switching, [ext]). */
static int digit_lo(orc_ctx* c, int j) { return j * c->alpha; }
static int digit_hi(orc_ctx* c, int j, int level) {
  int h = (j + 1) * c->alpha;
  return h < level ? h : level;
}

/* Galois element of a left rotation by r slots: 5^r mod 2N with r reduced
 * mod N/2 (5 has order N/2 in (Z/2N)^*). */
uint64_t orc_galois_elt(int log_n, int32_t r) {
  int64_t n_slots = (int64_t)1 << (log_n - 1);
  int64_t rr = ((r % n_slots) + n_slots) % n_slots;
  uint64_t m = (uint64_t)2 << log_n, k = 1;
  for (int64_t i = 0; i < rr; i++) k = (k * 5) % m;
  return k;
}

/* Automorphism X -> X^k on an evaluation-form polynomial: output slot j takes
 * input slot j' with 2*brv(j')+1 = (2*brv(j)+1)*k mod 2N, because
 * kappa_k(a)(psi^e) = a(psi^(e*k)). */
static void automorph_eval(orc_ctx* c, const uint64_t* in, uint64_t* out, uint64_t k) {
  uint32_t n = c->n;
  uint64_t m = 2 * (uint64_t)n;
  for (uint32_t j = 0; j < n; j++) {
    uint64_t e = 2 * (uint64_t)brv(j, c->log_n) + 1;
    uint64_t e2 = (e * k) % m;
    uint32_t jj = brv((uint32_t)((e2 - 1) / 2), c->log_n);
    out[j] = in[jj];
  }
}

/* Coefficient-form definition of the same automorphism:
 * a(X^k) = sum_i a_i X^(ik mod 2N), with X^N = -1. */
void orc_automorph_coef(const uint64_t* a, uint64_t* out, int log_n, uint64_t q, uint64_t k) {
  uint32_t n = 1u << log_n;
  uint64_t m = 2 * (uint64_t)n;
  for (uint32_t i = 0; i < n; i++) {
    uint64_t e = ((uint64_t)i * k) % m;
    if (e < n) out[e] = a[i] % q;
    else out[e - n] = submod(0, a[i] % q, q);
  }
}

void orc_automorph(orc_ctx* c, const uint64_t* in, uint64_t* out, int nlimbs, uint64_t k) {
  for (int t = 0; t < nlimbs; t++) automorph_eval(c, POLY(in, t, c->n), POLY(out, t, c->n), k);
}

/* (P - 1)/2 mod m, with P = product of the special primes (odd): computed as
 * (P mod m - 1) * 2^-1 mod m for odd m. */
static uint64_t P_mod(orc_ctx* c, uint64_t m);
static uint64_t half_P_mod(orc_ctx* c, uint64_t m) {
  uint64_t pm1 = submod(P_mod(c, m), 1, m);
  return mulmod(pm1, invmod(2, m), m);
}

/* P mod q_t, with P = product of the special primes. */
static uint64_t P_mod(orc_ctx* c, uint64_t m) {
  uint64_t r = 1 % m;
  for (int k = 0; k < c->alpha; k++) r = mulmod(r, c->q[c->L + k] % m, m);
  return r;
}

/* Hybrid evaluation key for s' (evaluation form over all np primes), [ext]
 * Han-Ki: digit j: b_j = -a_j s + e_j + P * [t in D_j] * s' on each limb t < L,
 * b_j = -a_j s + e_j on the special limbs; a_j uniform, drawn directly in
 * evaluation form; e_j discrete Gaussian.  Stream id = tag * 256 + j. */
static void gen_evk(orc_ctx* c, const uint64_t* sprime, uint32_t tag, uint64_t* key) {
  uint32_t n = c->n;
  int64_t* ec = malloc(sizeof(int64_t) * n);
  for (int j = 0; j < c->beta; j++) {
    uint32_t sid = tag * 256u + (uint32_t)j;
    for (uint32_t i = 0; i < n; i++) ec[i] = sample_gauss(c->seed, i, sid, DOM_EVK_E, c->gT, c->gK);
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < c->np; t++) {
      uint64_t* e = malloc(sizeof(uint64_t) * n);
      uint64_t q = c->q[t];
      uint64_t* b = key + ((size_t)(j * 2 + 0) * c->np + t) * n;
      uint64_t* a = key + ((size_t)(j * 2 + 1) * c->np + t) * n;
      for (uint32_t i = 0; i < n; i++) a[i] = sample_uniform(c->seed, i, (uint32_t)t, sid, DOM_EVK_A, q);
      for (uint32_t i = 0; i < n; i++) e[i] = smod(ec[i], q);
      ntt_limb(c, t, e);
      int in_digit = (t < c->L) && (t >= digit_lo(c, j)) && (t < digit_hi(c, j, c->L));
      uint64_t pm = P_mod(c, q);
      const uint64_t* s = POLY(c->s, t, n);
      const uint64_t* sp = POLY(sprime, t, n);
      for (uint32_t i = 0; i < n; i++) {
        uint64_t v = submod(e[i], mulmod(a[i], s[i], q), q);
        if (in_digit) v = addmod(v, mulmod(pm, sp[i], q), q);
        b[i] = v;
      }
      free(e);
    }
  }
  free(ec);
}

static size_t key_words(orc_ctx* c) { return (size_t)c->beta * 2 * c->np * c->n; }

void orc_destroy(orc_ctx* c) {
  if (!c) return;
  for (int t = 0; t < c->np; t++) { free(c->tw[t]); free(c->itw[t]); }
  free(c->s_coef); free(c->s); free(c->pk_b); free(c->pk_a); free(c->rlk);
  for (int i = 0; i < c->ngal; i++) free(c->gal[i].key);
  free(c->gal); free(c->cos_t); free(c->sin_t);
  free(c);
}

/* Key generation from the seed (Algorithm 2: the parameter server generates
 * pk and sk; Sec. 3: keys are ring elements).  Limb primes at limb_bits,
 * special primes at special_bits (distinct from the limbs). */
orc_ctx* orc_create(int log_n, int L, int limb_bits, int alpha, int special_bits, double scale,
                    double sigma, uint64_t seed, const int32_t* rots, int nrot) {
  if (log_n < 2 || log_n > 17 || L < 1 || alpha < 1 || L + alpha > ORC_MAX_PRIMES) return NULL;
  orc_ctx* c = calloc(1, sizeof(orc_ctx));
  c->log_n = log_n; c->n = 1 << log_n; c->L = L; c->alpha = alpha; c->np = L + alpha;
  c->beta = (L + alpha - 1) / alpha;
  c->scale = scale; c->sigma = sigma; c->seed = seed;
  uint32_t n = c->n;
  if (orc_gen_primes(limb_bits, log_n, L, NULL, 0, c->q) != L) { free(c); return NULL; }
  if (orc_gen_primes(special_bits, log_n, alpha, c->q, L, c->q + L) != alpha) { free(c); return NULL; }
  for (int t = 0; t < c->np; t++) {
    c->psi[t] = orc_min_root(c->q[t], log_n);
    c->tw[t] = malloc(sizeof(uint64_t) * n);
    c->itw[t] = malloc(sizeof(uint64_t) * n);
    make_tables(log_n, c->q[t], c->psi[t], c->tw[t], c->itw[t]);
    c->ninv[t] = invmod(n, c->q[t]);
  }
  c->gK = orc_gauss_table(sigma, c->gT);
  c->cos_t = malloc(sizeof(double) * 2 * n);
  c->sin_t = malloc(sizeof(double) * 2 * n);
  for (uint32_t t = 0; t < 2 * n; t++) {
    c->cos_t[t] = cos(M_PI * (double)t / (double)n);
    c->sin_t[t] = sin(M_PI * (double)t / (double)n);
  }
  /* secret s: ternary coefficients, stream (DOM_S, 0) */
  c->s_coef = malloc(n);
  c->s = malloc(sizeof(uint64_t) * (size_t)c->np * n);
  for (uint32_t i = 0; i < n; i++) c->s_coef[i] = (int8_t)sample_ternary(seed, i, 0, DOM_S);
  for (int t = 0; t < c->np; t++) {
    uint64_t* st = POLY(c->s, t, n);
    for (uint32_t i = 0; i < n; i++) st[i] = smod(c->s_coef[i], c->q[t]);
    ntt_limb(c, t, st);
  }
  /* public key (b, a) = (-a s + e, a) over the L limbs, a in evaluation form */
  c->pk_a = malloc(sizeof(uint64_t) * (size_t)L * n);
  c->pk_b = malloc(sizeof(uint64_t) * (size_t)L * n);
  {
    uint64_t* e = malloc(sizeof(uint64_t) * n);
    int64_t* ec = malloc(sizeof(int64_t) * n);
    for (uint32_t i = 0; i < n; i++) ec[i] = sample_gauss(seed, i, 0, DOM_PK_E, c->gT, c->gK);
    for (int t = 0; t < L; t++) {
      uint64_t q = c->q[t];
      uint64_t* a = POLY(c->pk_a, t, n);
      uint64_t* b = POLY(c->pk_b, t, n);
      for (uint32_t i = 0; i < n; i++) a[i] = sample_uniform(seed, i, (uint32_t)t, 0, DOM_PK_A, q);
      for (uint32_t i = 0; i < n; i++) e[i] = smod(ec[i], q);
      ntt_limb(c, t, e);
      const uint64_t* s = POLY(c->s, t, n);
      for (uint32_t i = 0; i < n; i++) b[i] = submod(e[i], mulmod(a[i], s[i], q), q);
    }
    free(e);
    free(ec);
  }
  /* relinearisation key: s' = s^2 */
  {
    uint64_t* s2 = malloc(sizeof(uint64_t) * (size_t)c->np * n);
    for (int t = 0; t < c->np; t++)
      for (uint32_t i = 0; i < n; i++)
        s2[(size_t)t * n + i] = mulmod(c->s[(size_t)t * n + i], c->s[(size_t)t * n + i], c->q[t]);
    c->rlk = malloc(sizeof(uint64_t) * key_words(c));
    gen_evk(c, s2, 0, c->rlk);
    free(s2);
  }
  /* rotation (Galois) keys: s' = kappa_k(s), tag = k */
  c->ngal = 0;
  c->gal = calloc(nrot > 0 ? nrot : 1, sizeof(orc_galkey));
  for (int r = 0; r < nrot; r++) {
    uint64_t k = orc_galois_elt(log_n, rots[r]);
    int dup = 0;
    for (int i = 0; i < c->ngal; i++)
      if (c->gal[i].gal == k) dup = 1;
    if (dup || k == 1) continue;
    uint64_t* sk = malloc(sizeof(uint64_t) * (size_t)c->np * n);
    orc_automorph(c, c->s, sk, c->np, k);
    orc_galkey* g = &c->gal[c->ngal++];
    g->step = rots[r];
    g->gal = k;
    g->key = malloc(sizeof(uint64_t) * key_words(c));
    gen_evk(c, sk, (uint32_t)k, g->key);
    free(sk);
  }
  return c;
}

void orc_get_primes(orc_ctx* c, uint64_t* out) { memcpy(out, c->q, sizeof(uint64_t) * c->np); }
void orc_get_roots(orc_ctx* c, uint64_t* out) { memcpy(out, c->psi, sizeof(uint64_t) * c->np); }
void orc_get_secret(orc_ctx* c, int8_t* out) { memcpy(out, c->s_coef, c->n); }
int orc_get_beta(orc_ctx* c) { return c->beta; }

/* Copies of the keys for the tests: which = 0 pk (b then a, [2][L][N]),
 * 1 relinearisation key, 2 + i Galois key i ([beta][2][np][N]). */
int orc_get_key(orc_ctx* c, int which, uint64_t* out) {
  size_t n = c->n;
  if (which == 0) {
    memcpy(out, c->pk_b, sizeof(uint64_t) * c->L * n);
    memcpy(out + c->L * n, c->pk_a, sizeof(uint64_t) * c->L * n);
    return 0;
  }
  if (which == 1) { memcpy(out, c->rlk, sizeof(uint64_t) * key_words(c)); return 0; }
  if (which - 2 < c->ngal) { memcpy(out, c->gal[which - 2].key, sizeof(uint64_t) * key_words(c)); return 0; }
  return -1;
}

/* ------------------------------------------------------------------------ */
/* Encode / decode (Sec. 3: canonical embedding).  Slot j <-> evaluation at   */
/* zeta_j = exp(i pi e_j / N), e_j = 5^j mod 2N, j < N/2.                    */
/* m_i = round((2 Delta / N) * sum_j Re(z_j * zeta_j^-i)), round half away.   */
/* ------------------------------------------------------------------------ */

/* Pre-rounding values (for tie analysis) and the rounded coefficients. */
void orc_encode_raw(orc_ctx* c, const double* re, const double* im, int nv, double scale,
                    double* raw) {
  uint32_t n = c->n, nh = n / 2;
  uint64_t m = 2 * (uint64_t)n;
  uint64_t* e = malloc(sizeof(uint64_t) * nh);
  uint64_t p = 1;
  for (uint32_t j = 0; j < nh; j++) { e[j] = p; p = (p * 5) % m; }
  for (uint32_t i = 0; i < n; i++) {
    double acc = 0.0;
    for (uint32_t j = 0; j < (uint32_t)nv && j < nh; j++) {
      uint64_t t = (e[j] * (uint64_t)i) % m;
      double zr = re ? re[j] : 0.0, zi = im ? im[j] : 0.0;
      acc += zr * c->cos_t[t] + zi * c->sin_t[t];
    }
    raw[i] = (2.0 * scale / (double)n) * acc;
  }
  free(e);
}

int orc_encode(orc_ctx* c, const double* re, const double* im, int nv, double scale, int64_t* out) {
  double* raw = malloc(sizeof(double) * c->n);
  orc_encode_raw(c, re, im, nv, scale, raw);
  int ok = 0;
  for (uint32_t i = 0; i < (uint32_t)c->n; i++) {
    if (!(fabs(raw[i]) < 9.2e18)) ok = -1;
    out[i] = (int64_t)llround(raw[i]);
  }
  free(raw);
  return ok;
}

/* z_j = (1/Delta) sum_i m_i zeta_j^i, from centered coefficients given as doubles. */
void orc_decode(orc_ctx* c, const double* mcoef, double scale, double* re, double* im) {
  uint32_t n = c->n, nh = n / 2;
  uint64_t m = 2 * (uint64_t)n, p = 1;
  for (uint32_t j = 0; j < nh; j++) {
    double ar = 0.0, ai = 0.0;
    for (uint32_t i = 0; i < n; i++) {
      uint64_t t = (p * (uint64_t)i) % m;
      ar += mcoef[i] * c->cos_t[t];
      ai += mcoef[i] * c->sin_t[t];
    }
    re[j] = ar / scale;
    if (im) im[j] = ai / scale;
    p = (p * 5) % m;
  }
}

/* ------------------------------------------------------------------------ */
/* Encrypt / decrypt (Sec. 3; Algorithm 1 uses pk, Algorithm 2 encrypts with  */
/* sk -- both are provided).  Ciphertexts are [2][level][N] evaluation form. */
/* ------------------------------------------------------------------------ */

int orc_encrypt(orc_ctx* c, const int64_t* msg, int level, int use_sk, uint32_t cid, uint64_t* ct) {
  if (level < 1 || level > c->L) return -1;
  uint32_t n = c->n;
  uint64_t* c0 = ct;
  uint64_t* c1 = ct + (size_t)level * n;
  uint64_t* t0 = malloc(sizeof(uint64_t) * n);
  uint64_t* t1 = malloc(sizeof(uint64_t) * n);
  uint64_t* tv = malloc(sizeof(uint64_t) * n);
  int64_t* e0 = malloc(sizeof(int64_t) * n);
  int64_t* e1 = malloc(sizeof(int64_t) * n);
  int8_t* v = malloc(n);
  for (uint32_t i = 0; i < n; i++) e0[i] = sample_gauss(c->seed, i, cid, DOM_ENC_E0, c->gT, c->gK);
  if (!use_sk) {
    for (uint32_t i = 0; i < n; i++) {
      v[i] = (int8_t)sample_ternary(c->seed, i, cid, DOM_ENC_V);
      e1[i] = sample_gauss(c->seed, i, cid, DOM_ENC_E1, c->gT, c->gK);
    }
  }
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    /* t0 = NTT(e0 + m) */
    for (uint32_t i = 0; i < n; i++) t0[i] = addmod(smod(e0[i], q), smod(msg[i], q), q);
    ntt_limb(c, t, t0);
    uint64_t* o0 = POLY(c0, t, n);
    uint64_t* o1 = POLY(c1, t, n);
    if (use_sk) {
      /* (-a s + e + m, a) */
      const uint64_t* s = POLY(c->s, t, n);
      for (uint32_t i = 0; i < n; i++) {
        uint64_t a = sample_uniform(c->seed, i, (uint32_t)t, cid, DOM_ENC_A, q);
        o1[i] = a;
        o0[i] = submod(t0[i], mulmod(a, s[i], q), q);
      }
    } else {
      /* (v b + e0 + m, v a + e1) */
      for (uint32_t i = 0; i < n; i++) tv[i] = smod(v[i], q);
      ntt_limb(c, t, tv);
      for (uint32_t i = 0; i < n; i++) t1[i] = smod(e1[i], q);
      ntt_limb(c, t, t1);
      const uint64_t* b = POLY(c->pk_b, t, n);
      const uint64_t* a = POLY(c->pk_a, t, n);
      for (uint32_t i = 0; i < n; i++) {
        o0[i] = addmod(mulmod(tv[i], b[i], q), t0[i], q);
        o1[i] = addmod(mulmod(tv[i], a[i], q), t1[i], q);
      }
    }
  }
  free(t0); free(t1); free(tv); free(e0); free(e1); free(v);
  return 0;
}

/* Little bignum: little-endian 64-bit words. */
#define BN_W 32
typedef struct { uint64_t w[BN_W]; } bn;

static void bn_mul_small_add(bn* x, uint64_t m, uint64_t a) {
  u128 carry = a;
  for (int i = 0; i < BN_W; i++) {
    u128 v = (u128)x->w[i] * m + carry;
    x->w[i] = (uint64_t)v;
    carry = v >> 64;
  }
}
static int bn_cmp(const bn* a, const bn* b) {
  for (int i = BN_W - 1; i >= 0; i--) {
    if (a->w[i] != b->w[i]) return a->w[i] < b->w[i] ? -1 : 1;
  }
  return 0;
}
static void bn_sub(bn* a, const bn* b) { /* a -= b, a >= b */
  uint64_t borrow = 0;
  for (int i = 0; i < BN_W; i++) {
    u128 v = (u128)a->w[i] - b->w[i] - borrow;
    a->w[i] = (uint64_t)v;
    borrow = (uint64_t)(v >> 64) ? 1 : 0;
  }
}
static double bn_to_double(const bn* a) {
  double r = 0.0;
  for (int i = BN_W - 1; i >= 0; i--) r = r * 18446744073709551616.0 + (double)a->w[i];
  return r;
}

/* CRT of residues r[0..level-1] (one coefficient) to the centered integer in
 * (-Q/2, Q/2], by Garner's mixed-radix digits.  Returns sign and magnitude. */
static void crt_centered(orc_ctx* c, const uint64_t* r, int level, bn* mag, int* neg) {
  uint64_t d[ORC_MAX_PRIMES];
  for (int i = 0; i < level; i++) {
    /* d_i = (r_i - (d_0 + d_1 q_0 + ... )) / (q_0 ... q_{i-1}) mod q_i */
    uint64_t qi = c->q[i], acc = 0, prod = 1 % qi;
    for (int k = 0; k < i; k++) {
      acc = addmod(acc, mulmod(d[k] % qi, prod, qi), qi);
      prod = mulmod(prod, c->q[k] % qi, qi);
    }
    d[i] = mulmod(submod(r[i] % qi, acc, qi), invmod(prod, qi), qi);
  }
  bn v; memset(&v, 0, sizeof v);
  for (int i = level - 1; i >= 0; i--) bn_mul_small_add(&v, c->q[i], d[i]); /* Horner */
  bn Q; memset(&Q, 0, sizeof Q); Q.w[0] = 1;
  for (int i = 0; i < level; i++) bn_mul_small_add(&Q, c->q[i], 0);
  bn half; /* floor(Q/2): a one-bit right shift across the words */
  for (int i = 0; i < BN_W; i++) {
    uint64_t hi = (i + 1 < BN_W) ? Q.w[i + 1] : 0;
    half.w[i] = (Q.w[i] >> 1) | (hi << 63);
  }
  if (bn_cmp(&v, &half) > 0) { bn t = Q; bn_sub(&t, &v); *mag = t; *neg = 1; }
  else { *mag = v; *neg = 0; }
}

/* m = c0 + c1 s over `level` limbs, back to coefficients, CRT-centered.
 * Outputs the centered coefficients as doubles; if `words` is non-NULL also
 * the exact magnitudes ([N][nw] little-endian words) and signs. */
int orc_decrypt(orc_ctx* c, const uint64_t* ct, int level, double* out, uint64_t* words, int nw,
                int8_t* signs) {
  if (level < 1 || level > c->L) return -1;
  uint32_t n = c->n;
  uint64_t* m = malloc(sizeof(uint64_t) * (size_t)level * n);
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    const uint64_t* c0 = POLY(ct, t, n);
    const uint64_t* c1 = POLY(ct + (size_t)level * n, t, n);
    const uint64_t* s = POLY(c->s, t, n);
    uint64_t* mt = POLY(m, t, n);
    for (uint32_t i = 0; i < n; i++) mt[i] = addmod(c0[i], mulmod(c1[i], s[i], q), q);
    intt_limb(c, t, mt);
  }
  uint64_t r[ORC_MAX_PRIMES];
  for (uint32_t i = 0; i < n; i++) {
    for (int t = 0; t < level; t++) r[t] = m[(size_t)t * n + i];
    bn mag; int neg;
    crt_centered(c, r, level, &mag, &neg);
    double v = bn_to_double(&mag);
    out[i] = neg ? -v : v;
    if (words) {
      for (int k = 0; k < nw; k++) words[(size_t)i * nw + k] = k < BN_W ? mag.w[k] : 0;
      signs[i] = (int8_t)neg;
    }
  }
  free(m);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Homomorphic operations (Sec. 3: addition, multiplication, rescaling;      */
/* Eq. 1-2: the encrypted op must decrypt to the plaintext op).              */
/* ------------------------------------------------------------------------ */

/* a + b at a common level (both already at `level`). */
void orc_add(orc_ctx* c, const uint64_t* a, const uint64_t* b, int level, uint64_t* out) {
  uint32_t n = c->n;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < level; t++) {
      size_t off = ((size_t)p * level + t) * n;
      for (uint32_t i = 0; i < n; i++) out[off + i] = addmod(a[off + i], b[off + i], c->q[t]);
    }
}

void orc_sub(orc_ctx* c, const uint64_t* a, const uint64_t* b, int level, uint64_t* out) {
  uint32_t n = c->n;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < level; t++) {
      size_t off = ((size_t)p * level + t) * n;
      for (uint32_t i = 0; i < n; i++) out[off + i] = submod(a[off + i], b[off + i], c->q[t]);
    }
}

/* Dropping limbs (modulus reduction without division): keep limbs < to. */
void orc_drop(orc_ctx* c, const uint64_t* a, int level, int to, uint64_t* out) {
  uint32_t n = c->n;
  for (int p = 0; p < 2; p++)
    memmove(out + (size_t)p * to * n, a + (size_t)p * level * n, sizeof(uint64_t) * (size_t)to * n);
}

/* Multiplication by an integer constant c (the constant polynomial). */
void orc_mul_int(orc_ctx* c, const uint64_t* a, int level, int64_t k, uint64_t* out) {
  uint32_t n = c->n;
  for (int p = 0; p < 2; p++)
    for (int t = 0; t < level; t++) {
      uint64_t kt = smod(k, c->q[t]);
      size_t off = ((size_t)p * level + t) * n;
      for (uint32_t i = 0; i < n; i++) out[off + i] = mulmod(a[off + i], kt, c->q[t]);
    }
}

/* Addition of an integer constant polynomial k: its evaluations are all k,
 * so k is added to every evaluation of c0. */
void orc_add_int(orc_ctx* c, const uint64_t* a, int level, int64_t k, uint64_t* out) {
  uint32_t n = c->n;
  memmove(out, a, sizeof(uint64_t) * 2 * (size_t)level * n);
  for (int t = 0; t < level; t++) {
    uint64_t kt = smod(k, c->q[t]);
    for (uint32_t i = 0; i < n; i++) out[(size_t)t * n + i] = addmod(out[(size_t)t * n + i], kt, c->q[t]);
  }
}

/* Multiplication by a plaintext given as integer coefficients. */
void orc_mul_plain(orc_ctx* c, const uint64_t* a, int level, const int64_t* m, uint64_t* out) {
  uint32_t n = c->n;
  uint64_t* pt = malloc(sizeof(uint64_t) * n);
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    for (uint32_t i = 0; i < n; i++) pt[i] = smod(m[i], q);
    ntt_limb(c, t, pt);
    for (int p = 0; p < 2; p++) {
      size_t off = ((size_t)p * level + t) * n;
      for (uint32_t i = 0; i < n; i++) out[off + i] = mulmod(a[off + i], pt[i], q);
    }
  }
  free(pt);
}

/* Tensor product: (d0, d1, d2) = (a0 b0, a0 b1 + a1 b0, a1 b1); out [3][level][N]. */
void orc_tensor(orc_ctx* c, const uint64_t* a, const uint64_t* b, int level, uint64_t* out) {
  uint32_t n = c->n;
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    const uint64_t* a0 = POLY(a, t, n); const uint64_t* a1 = POLY(a, level + t, n);
    const uint64_t* b0 = POLY(b, t, n); const uint64_t* b1 = POLY(b, level + t, n);
    uint64_t* d0 = POLY(out, t, n); uint64_t* d1 = POLY(out, level + t, n);
    uint64_t* d2 = POLY(out, 2 * level + t, n);
    for (uint32_t i = 0; i < n; i++) {
      d0[i] = mulmod(a0[i], b0[i], q);
      d1[i] = addmod(mulmod(a0[i], b1[i], q), mulmod(a1[i], b0[i], q), q);
      d2[i] = mulmod(a1[i], b1[i], q);
    }
  }
}

/* ModUp of digit j [ext]: for x given by its coefficient residues on the
 * digit's limbs D_j, the approximate basis conversion
 *   y_c = sum_{i in D_j} [x_i * (Q_j/q_i)^-1]_{q_i} * (Q_j/q_i mod c)  mod c
 * (residues taken in [0, q_i); no exact-CRT correction).  `xcoef` holds
 * coefficient residues of all limbs [level][N]; target prime index tp. */
static void modup_limb(orc_ctx* c, const uint64_t* xcoef, int level, int j, int tp, uint64_t* y) {
  uint32_t n = c->n;
  int lo = digit_lo(c, j), hi = digit_hi(c, j, level);
  uint64_t qc = c->q[tp];
  for (uint32_t k = 0; k < n; k++) y[k] = 0;
  for (int i = lo; i < hi; i++) {
    uint64_t qi = c->q[i];
    uint64_t qhat_i = 1 % qi, qhat_c = 1 % qc; /* Q_j/q_i mod q_i and mod c */
    for (int i2 = lo; i2 < hi; i2++) {
      if (i2 == i) continue;
      qhat_i = mulmod(qhat_i, c->q[i2] % qi, qi);
      qhat_c = mulmod(qhat_c, c->q[i2] % qc, qc);
    }
    uint64_t qhat_inv = invmod(qhat_i, qi);
    const uint64_t* x = POLY(xcoef, i, n);
    for (uint32_t k = 0; k < n; k++) {
      uint64_t u = mulmod(x[k], qhat_inv, qi);
      y[k] = addmod(y[k], mulmod(u % qc, qhat_c, qc), qc);
    }
  }
}

/* Exposed for the exact big-integer pins: ModUp of digit j of coefficient
 * residues xcoef [level][N] onto prime index tp; result in coefficient form. */
void orc_modup_coef(orc_ctx* c, const uint64_t* xcoef, int level, int j, int tp, uint64_t* y) {
  modup_limb(c, xcoef, level, j, tp, y);
}

static uint64_t bn_mod_small(const bn* a, uint64_t m) {
  u128 r = 0;
  for (int i = BN_W - 1; i >= 0; i--) r = ((r << 64) | a->w[i]) % m;
  return (uint64_t)r;
}

/* ModDown conversion [ext]: the exact basis conversion from the special basis
 * P to prime q_t of coefficient residues ycoefP [alpha][N]: the integer
 * Y in [0, P) with Y = y_k mod p_k for every k (CRT by Garner's mixed-radix
 * digits), reduced mod q_t.  Exact, so that the division by P that follows
 * rounds every coefficient (with one special prime Y = y_0). */
static void moddown_conv(orc_ctx* c, const uint64_t* ycoefP, int t, uint64_t* out) {
  uint32_t n = c->n;
  int a = c->alpha;
  const uint64_t* ps = c->q + c->L;
  for (uint32_t i = 0; i < n; i++) {
    uint64_t d[ORC_MAX_PRIMES];
    for (int k = 0; k < a; k++) {
      /* d_k = (y_k - (d_0 + d_1 p_0 + ...)) / (p_0 ... p_{k-1}) mod p_k */
      uint64_t pk = ps[k], acc = 0, prod = 1 % pk;
      for (int k2 = 0; k2 < k; k2++) {
        acc = addmod(acc, mulmod(d[k2] % pk, prod, pk), pk);
        prod = mulmod(prod, ps[k2] % pk, pk);
      }
      d[k] = mulmod(submod(ycoefP[(size_t)k * n + i] % pk, acc, pk), invmod(prod, pk), pk);
    }
    bn y;
    memset(&y, 0, sizeof y);
    for (int k = a - 1; k >= 0; k--) bn_mul_small_add(&y, ps[k], d[k]); /* Horner */
    out[i] = bn_mod_small(&y, c->q[t]);
  }
}

void orc_moddown_conv(orc_ctx* c, const uint64_t* ycoefP, int t, uint64_t* out) {
  moddown_conv(c, ycoefP, t, out);
}

static const uint64_t* find_key(orc_ctx* c, int key_id) {
  if (key_id < 0) return c->rlk;
  if (key_id < c->ngal) return c->gal[key_id].key;
  return NULL;
}

/* ModDown of a key switch's two accumulators acc [2][level + alpha][N]
 * (evaluation form over Q_level and P) to (k0, k1) [level][N]: division by P
 * with rounding, as described at keyswitch below. */
static void moddown_pair(orc_ctx* c, const uint64_t* acc, int level, uint64_t* k0, uint64_t* k1) {
  uint32_t n = c->n;
  int nt = level + c->alpha;
  uint64_t* yP = malloc(sizeof(uint64_t) * (size_t)c->alpha * n);
  uint64_t* conv = malloc(sizeof(uint64_t) * n);
  for (int p = 0; p < 2; p++) {
    const uint64_t* ap = acc + (size_t)p * nt * n;
    for (int k = 0; k < c->alpha; k++) {
      uint64_t pk = c->q[c->L + k];
      uint64_t hk = half_P_mod(c, pk);
      memcpy(POLY(yP, k, n), POLY(ap, level + k, n), sizeof(uint64_t) * n);
      intt_limb(c, c->L + k, POLY(yP, k, n));
      for (uint32_t i = 0; i < n; i++) yP[(size_t)k * n + i] = addmod(yP[(size_t)k * n + i], hk, pk);
    }
    uint64_t* dst = p == 0 ? k0 : k1;
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < level; t++) {
      uint64_t* cv = malloc(sizeof(uint64_t) * n);
      uint64_t q = c->q[t];
      uint64_t ht = half_P_mod(c, q);
      moddown_conv(c, yP, t, cv);
      for (uint32_t i = 0; i < n; i++) cv[i] = submod(cv[i], ht, q);
      ntt_limb(c, t, cv);
      uint64_t pinv = invmod(P_mod(c, q), q);
      const uint64_t* at = POLY(ap, t, n);
      uint64_t* o = POLY(dst, t, n);
      for (uint32_t i = 0; i < n; i++) o[i] = mulmod(submod(at[i], cv[i], q), pinv, q);
      free(cv);
    }
  }
  free(yP); free(conv);
}

/* Hybrid key switching [ext], at `level`: input d (evaluation form [level][N]),
 * key for s' -> s; output (k0, k1) [level][N] each, with k0 + k1 s ~ d s'.
 * Steps in order: d to coefficients; per digit ModUp to Q_level + P and back
 * to evaluation form; inner product with the key; ModDown with rounding
 * (division by P rounds, as the rescale does -- Sec. 3's "homomorphic
 * rounding"; flooring would leave a -1/2 bias on every coefficient of both
 * parts, which concentrates in the lowest-frequency slot):
 *   y = INTT_P(acc_P) + h (every coefficient),  h = (P-1)/2,
 *   out_t = (acc_t - NTT_t(Conv_{P->q_t}(y) - h)) * P^-1  mod q_t,
 * with the exact conversion Conv (the lift of y to [0, P)), i.e.
 * out = round(acc / P): Conv(y) - h is the centered residue of acc mod P.  An
 * approximate conversion would add v P, 0 <= v < alpha, and so a one-sided
 * error of -v on every coefficient, the same drift as flooring. */
/* The inner products of a key switch before its ModDown: acc [2][level +
 * alpha][N] (evaluation form over Q_level and P, zeroed by the caller) +=
 * sum_j ModUp_j(d) * key_j.  Used by keyswitch below and, with the ModDown
 * merged into the rescale, by the multiplication. */
static void ks_inner(orc_ctx* c, const uint64_t* d, int level, const uint64_t* key, uint64_t* acc) {
  uint32_t n = c->n;
  int nt = level + c->alpha; /* target primes: limbs 0..level-1, specials L..L+alpha-1 */
  int beta_l = (level + c->alpha - 1) / c->alpha;
  uint64_t* dc = malloc(sizeof(uint64_t) * (size_t)level * n);
  for (int t = 0; t < level; t++) {
    memcpy(POLY(dc, t, n), POLY(d, t, n), sizeof(uint64_t) * n);
    intt_limb(c, t, POLY(dc, t, n));
  }
  for (int j = 0; j < beta_l; j++) {
#pragma omp parallel for schedule(dynamic)
    for (int ti = 0; ti < nt; ti++) {
      uint64_t* ext = malloc(sizeof(uint64_t) * n);
      int tp = ti < level ? ti : c->L + (ti - level); /* prime index */
      uint64_t q = c->q[tp];
      if (tp < level && tp >= digit_lo(c, j) && tp < digit_hi(c, j, level)) {
        memcpy(ext, POLY(d, tp, n), sizeof(uint64_t) * n); /* exact on the digit's own limbs */
      } else {
        modup_limb(c, dc, level, j, tp, ext);
        ntt_limb(c, tp, ext);
      }
      const uint64_t* kb = key + ((size_t)(j * 2 + 0) * c->np + tp) * n;
      const uint64_t* ka = key + ((size_t)(j * 2 + 1) * c->np + tp) * n;
      uint64_t* a0 = POLY(acc, ti, n);
      uint64_t* a1 = POLY(acc, nt + ti, n);
      for (uint32_t i = 0; i < n; i++) {
        a0[i] = addmod(a0[i], mulmod(ext[i], kb[i], q), q);
        a1[i] = addmod(a1[i], mulmod(ext[i], ka[i], q), q);
      }
      free(ext);
    }
  }
  free(dc);
}

static void keyswitch(orc_ctx* c, const uint64_t* d, int level, const uint64_t* key,
                      uint64_t* k0, uint64_t* k1) {
  uint64_t* acc = calloc((size_t)2 * (level + c->alpha) * c->n, sizeof(uint64_t)); /* [2][nt][N] */
  ks_inner(c, d, level, key, acc);
  moddown_pair(c, acc, level, k0, k1);
  free(acc);
}

/* Exact conversion from k primes pr[0..k) to modulus m of coefficient
 * residues y [k][N]: the integer Y in [0, prod pr) with Y = y_u mod pr[u]
 * (Garner's mixed-radix digits), reduced mod m. */
static void conv_exact(const uint64_t* y, const uint64_t* pr, int k, uint32_t n, uint64_t m, uint64_t* out) {
  for (uint32_t i = 0; i < n; i++) {
    uint64_t dg[ORC_MAX_PRIMES];
    for (int u = 0; u < k; u++) {
      uint64_t pu = pr[u], acc = 0, prod = 1 % pu;
      for (int v = 0; v < u; v++) {
        acc = addmod(acc, mulmod(dg[v] % pu, prod, pu), pu);
        prod = mulmod(prod, pr[v] % pu, pu);
      }
      dg[u] = mulmod(submod(y[(size_t)u * n + i] % pu, acc, pu), invmod(prod, pu), pu);
    }
    bn Y;
    memset(&Y, 0, sizeof Y);
    for (int u = k - 1; u >= 0; u--) bn_mul_small_add(&Y, pr[u], dg[u]);
    out[i] = bn_mod_small(&Y, m);
  }
}

/* The ModDown of a relinearisation merged with the rescale that follows it
 * [ext]: one division with rounding by P q_{level-1} of
 *   V = P (d0, d1) + acc     over Q_level * P
 * (acc [2][level + alpha][N] the key switch's inner products, d01
 * [2][level][N] the tensor's first two parts, both evaluation form), instead
 * of dividing acc by P, adding d and dividing by q_{level-1}.  V's residues
 * on the dropped primes are acc's on p_k (P d vanishes there) and
 * acc_{level-1} + P d_{level-1} on q_{level-1}; with Y their exact lift plus
 * h = (P q_{level-1} - 1)/2 (coefficient form),
 *   out_t = (V_t - NTT_t(Y mod q_t - h)) * (P q_{level-1})^-1   (t < level-1),
 * i.e. out = round(V / (P q_{level-1})).  out [2][level-1][N]. */
static void moddown_rescale_pair(orc_ctx* c, const uint64_t* acc, const uint64_t* d01, int level, uint64_t* out) {
  uint32_t n = c->n;
  int a = c->alpha, nt = level + a, l = level - 1, k = a + 1;
  uint64_t pr[ORC_MAX_PRIMES];
  pr[0] = c->q[l];
  for (int u = 0; u < a; u++) pr[1 + u] = c->q[c->L + u];
  uint64_t* y = malloc(sizeof(uint64_t) * (size_t)k * n);
  uint64_t* conv = malloc(sizeof(uint64_t) * n);
  uint64_t* res = malloc(sizeof(uint64_t) * 2 * (size_t)l * n);
  for (int p = 0; p < 2; p++) {
    const uint64_t* ap = acc + (size_t)p * nt * n;
    const uint64_t* dp = d01 + (size_t)p * level * n;
    for (int u = 0; u < k; u++) {
      uint64_t m = pr[u];
      uint64_t* yu = POLY(y, u, n);
      if (u == 0) {
        uint64_t Pm = P_mod(c, m);
        for (uint32_t i = 0; i < n; i++) yu[i] = addmod(ap[(size_t)l * n + i], mulmod(Pm, dp[(size_t)l * n + i], m), m);
        intt_limb(c, l, yu);
      } else {
        memcpy(yu, POLY(ap, level + u - 1, n), sizeof(uint64_t) * n);
        intt_limb(c, c->L + u - 1, yu);
      }
      /* + h mod m, h = (P q_l - 1)/2 */
      uint64_t h = mulmod(submod(mulmod(P_mod(c, m), pr[0] % m, m), 1, m), invmod(2, m), m);
      for (uint32_t i = 0; i < n; i++) yu[i] = addmod(yu[i], h, m);
    }
#pragma omp parallel for schedule(dynamic)
    for (int t = 0; t < l; t++) {
      uint64_t* cv = malloc(sizeof(uint64_t) * n);
      uint64_t q = c->q[t];
      uint64_t Pq = mulmod(P_mod(c, q), pr[0] % q, q);
      uint64_t ht = mulmod(submod(Pq, 1, q), invmod(2, q), q);
      conv_exact(y, pr, k, n, q, cv);
      for (uint32_t i = 0; i < n; i++) cv[i] = submod(cv[i], ht, q);
      ntt_limb(c, t, cv);
      uint64_t inv = invmod(Pq, q), Pm = P_mod(c, q);
      uint64_t* o = POLY(res, p * l + t, n);
      for (uint32_t i = 0; i < n; i++) {
        uint64_t v = addmod(ap[(size_t)t * n + i], mulmod(Pm, dp[(size_t)t * n + i], q), q);
        o[i] = mulmod(submod(v, cv[i], q), inv, q);
      }
      free(cv);
    }
  }
  memcpy(out, res, sizeof(uint64_t) * 2 * (size_t)l * n);
  free(y); free(conv); free(res);
}

/* The two ModDown forms above on accumulators the caller gives (boundary
 * tests feed P-parts whose lift lies next to 0 or P): acc [2][level +
 * alpha][N], d01 [2][level][N], evaluation form. */
int orc_moddown(orc_ctx* c, const uint64_t* acc, int level, uint64_t* k0, uint64_t* k1) {
  if (level < 1 || level > c->L) return -1;
  moddown_pair(c, acc, level, k0, k1);
  return 0;
}

int orc_moddown_rescale(orc_ctx* c, const uint64_t* acc, const uint64_t* d01, int level, uint64_t* out) {
  if (level < 2 || level > c->L) return -1;
  moddown_rescale_pair(c, acc, d01, level, out);
  return 0;
}

/* key_id: -1 relinearisation key, i >= 0 Galois key i (in creation order). */
int orc_keyswitch(orc_ctx* c, const uint64_t* d, int level, int key_id, uint64_t* k0, uint64_t* k1) {
  const uint64_t* key = find_key(c, key_id);
  if (!key || level < 1 || level > c->L) return -1;
  keyswitch(c, d, level, key, k0, k1);
  return 0;
}

/* Rescale by the last limb q_last = q[level-1] (Sec. 2-3: "homomorphic
 * rounding"): out = round(c / q_last) residue-wise.  With r the centered
 * representative of c mod q_last (|r| <= (q_last-1)/2), c - r is divisible by
 * q_last and (c - r)/q_last = round(c/q_last):
 *   out_t = (c_t - NTT_t(r mod q_t)) * q_last^-1  mod q_t,  t < level - 1. */
int orc_rescale(orc_ctx* c, const uint64_t* a, int level, uint64_t* out) {
  if (level < 2) return -1;
  uint32_t n = c->n;
  int lt = level - 1;
  uint64_t ql = c->q[lt], half = (ql - 1) / 2;
  uint64_t* last = malloc(sizeof(uint64_t) * n);
  uint64_t* rt = malloc(sizeof(uint64_t) * n);
  uint64_t* res = malloc(sizeof(uint64_t) * 2 * (size_t)lt * n);
  for (int p = 0; p < 2; p++) {
    memcpy(last, POLY(a, p * level + lt, n), sizeof(uint64_t) * n);
    intt_limb(c, lt, last);
    for (int t = 0; t < lt; t++) {
      uint64_t q = c->q[t];
      for (uint32_t i = 0; i < n; i++) {
        int64_t r = last[i] > half ? (int64_t)last[i] - (int64_t)ql : (int64_t)last[i];
        rt[i] = smod(r, q);
      }
      ntt_limb(c, t, rt);
      uint64_t inv = invmod(ql % q, q);
      const uint64_t* at = POLY(a, p * level + t, n);
      uint64_t* o = POLY(res, p * lt + t, n);
      for (uint32_t i = 0; i < n; i++) o[i] = mulmod(submod(at[i], rt[i], q), inv, q);
    }
  }
  memcpy(out, res, sizeof(uint64_t) * 2 * (size_t)lt * n);
  free(last); free(rt); free(res);
  return 0;
}

/* Relinearise a three-part ciphertext d = (d0, d1, d2) [3][level][N] and
 * rescale: the inner products of d2 with the s^2 key, then the division of
 * P (d0, d1) + acc by P q_{level-1} with one rounding (moddown_rescale_pair).
 * out has level - 1 limbs. */
static void relin_rescale(orc_ctx* c, const uint64_t* d, int level, uint64_t* out) {
  uint64_t* acc = calloc((size_t)2 * (level + c->alpha) * c->n, sizeof(uint64_t));
  ks_inner(c, POLY(d, 2 * level, c->n), level, c->rlk, acc);
  moddown_rescale_pair(c, acc, d, level, out);
  free(acc);
}

/* HMult: tensor, relinearise d2 with the s^2 key and rescale, the key
 * switch's division by P and the rescale's by q[level-1] taken as one
 * rounding (relin_rescale).  out has level - 1 limbs.  scale_out = scale_a *
 * scale_b / q[level-1]. */
int orc_mul_relin_rescale(orc_ctx* c, const uint64_t* a, const uint64_t* b, int level, uint64_t* out) {
  if (level < 2 || level > c->L) return -1;
  uint32_t n = c->n;
  uint64_t* d = malloc(sizeof(uint64_t) * 3 * (size_t)level * n);
  orc_tensor(c, a, b, level, d);
  relin_rescale(c, d, level, out);
  free(d);
  return 0;
}

/* Multiplication + relinearisation without rescale (out has `level` limbs). */
int orc_mul_relin(orc_ctx* c, const uint64_t* a, const uint64_t* b, int level, uint64_t* out) {
  if (level < 1 || level > c->L) return -1;
  uint32_t n = c->n;
  uint64_t* d = malloc(sizeof(uint64_t) * 3 * (size_t)level * n);
  uint64_t* k0 = malloc(sizeof(uint64_t) * (size_t)level * n);
  uint64_t* k1 = malloc(sizeof(uint64_t) * (size_t)level * n);
  orc_tensor(c, a, b, level, d);
  keyswitch(c, POLY(d, 2 * level, n), level, c->rlk, k0, k1);
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    for (uint32_t i = 0; i < n; i++) {
      out[(size_t)t * n + i] = addmod(d[(size_t)t * n + i], k0[(size_t)t * n + i], q);
      out[((size_t)level + t) * n + i] = addmod(d[((size_t)level + t) * n + i], k1[(size_t)t * n + i], q);
    }
  }
  free(d); free(k0); free(k1);
  return 0;
}

static int find_gal(orc_ctx* c, uint64_t k) {
  for (int i = 0; i < c->ngal; i++)
    if (c->gal[i].gal == k) return i;
  return -1;
}

/* Rotation by r slots (slot j <- slot j + r) [ext]: apply kappa_k, k = 5^r,
 * to both parts, then switch kappa_k(c1) from kappa_k(s) back to s. */
int orc_rotate(orc_ctx* c, const uint64_t* a, int level, int32_t r, uint64_t* out) {
  uint32_t n = c->n;
  uint64_t k = orc_galois_elt(c->log_n, r);
  if (k == 1) { memmove(out, a, sizeof(uint64_t) * 2 * (size_t)level * n); return 0; }
  int gi = find_gal(c, k);
  if (gi < 0) return -2;
  uint64_t* t0 = malloc(sizeof(uint64_t) * (size_t)level * n);
  uint64_t* t1 = malloc(sizeof(uint64_t) * (size_t)level * n);
  uint64_t* k0 = malloc(sizeof(uint64_t) * (size_t)level * n);
  uint64_t* k1 = malloc(sizeof(uint64_t) * (size_t)level * n);
  orc_automorph(c, a, t0, level, k);
  orc_automorph(c, a + (size_t)level * n, t1, level, k);
  keyswitch(c, t1, level, c->gal[gi].key, k0, k1);
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    for (uint32_t i = 0; i < n; i++) {
      out[(size_t)t * n + i] = addmod(t0[(size_t)t * n + i], k0[(size_t)t * n + i], q);
      out[((size_t)level + t) * n + i] = k1[(size_t)t * n + i];
    }
  }
  free(t0); free(t1); free(k0); free(k1);
  return 0;
}

/* Sum of rotations with one shared decomposition (hoisting) [ext]:
 *   out = a + sum_{s < ns} rot(a, r_s),   k_s = 5^{r_s} mod 2N.
 * The paper leaves the evaluation of rotations to HEAAN; this is the standard
 * hoisted form of a rotate-and-sum.  The digits of a1 are raised once,
 *   y_j = ModUp_j(a1)  (coefficient form over Q_level and P; on the digit's
 *                       own limbs the limb itself),
 * rotation s takes kappa_{k_s}(y_j) (the coefficient automorphism applied to
 * every limb) as its extended digit, the inner products of all rotations with
 * their Galois keys are summed over Q_level * P, and one ModDown (division by
 * P with rounding, as in keyswitch) gives (k0, k1):
 *   out0 = a0 + sum_s kappa_{k_s}(a0) + k0,   out1 = a1 + k1.
 * The approximate conversion is not odd (it maps -x to |D_j| Q_j - y, not to
 * -y), so kappa(y_j) and ModUp_j(kappa(a1)) may differ by multiples of Q_j:
 * the result encrypts the same sum as rotating and adding one at a time, with
 * residues of its own.  Returns -2 when a Galois key is missing, -3 for a
 * rotation by 0 slots. */
#define ORC_MAX_ROT 16
int orc_rotate_sum(orc_ctx* c, const uint64_t* a, int level, const int32_t* steps, int ns, uint64_t* out) {
  uint32_t n = c->n;
  if (level < 1 || level > c->L || ns < 1 || ns > ORC_MAX_ROT) return -1;
  int nt = level + c->alpha, beta_l = (level + c->alpha - 1) / c->alpha;
  uint64_t ks[ORC_MAX_ROT];
  const uint64_t* keys[ORC_MAX_ROT];
  for (int s = 0; s < ns; s++) {
    ks[s] = orc_galois_elt(c->log_n, steps[s]);
    if (ks[s] == 1) return -3;
    int gi = find_gal(c, ks[s]);
    if (gi < 0) return -2;
    keys[s] = c->gal[gi].key;
  }
  const uint64_t* a0 = a;
  const uint64_t* a1 = a + (size_t)level * n;
  uint64_t* dc = malloc(sizeof(uint64_t) * (size_t)level * n);
  for (int t = 0; t < level; t++) {
    memcpy(POLY(dc, t, n), POLY(a1, t, n), sizeof(uint64_t) * n);
    intt_limb(c, t, POLY(dc, t, n));
  }
  uint64_t* acc = calloc((size_t)2 * nt * n, sizeof(uint64_t)); /* [2][nt][N], summed over rotations */
  for (int j = 0; j < beta_l; j++) {
#pragma omp parallel for schedule(dynamic)
    for (int ti = 0; ti < nt; ti++) {
      uint64_t* y = malloc(sizeof(uint64_t) * n);
      uint64_t* z = malloc(sizeof(uint64_t) * n);
      int tp = ti < level ? ti : c->L + (ti - level);
      uint64_t q = c->q[tp];
      if (tp < level && tp >= digit_lo(c, j) && tp < digit_hi(c, j, level))
        memcpy(y, POLY(dc, tp, n), sizeof(uint64_t) * n);
      else
        modup_limb(c, dc, level, j, tp, y);
      for (int s = 0; s < ns; s++) {
        orc_automorph_coef(y, z, c->log_n, q, ks[s]);
        ntt_limb(c, tp, z);
        const uint64_t* kb = keys[s] + ((size_t)(j * 2 + 0) * c->np + tp) * n;
        const uint64_t* ka = keys[s] + ((size_t)(j * 2 + 1) * c->np + tp) * n;
        uint64_t* s0 = POLY(acc, ti, n);
        uint64_t* s1 = POLY(acc, nt + ti, n);
        for (uint32_t i = 0; i < n; i++) {
          s0[i] = addmod(s0[i], mulmod(z[i], kb[i], q), q);
          s1[i] = addmod(s1[i], mulmod(z[i], ka[i], q), q);
        }
      }
      free(y); free(z);
    }
  }
  uint64_t* z = malloc(sizeof(uint64_t) * n);
  uint64_t* k0 = malloc(sizeof(uint64_t) * (size_t)level * n);
  uint64_t* k1 = malloc(sizeof(uint64_t) * (size_t)level * n);
  moddown_pair(c, acc, level, k0, k1);
  uint64_t* res = malloc(sizeof(uint64_t) * 2 * (size_t)level * n);
  for (int t = 0; t < level; t++) {
    uint64_t q = c->q[t];
    uint64_t* r0 = POLY(res, t, n);
    uint64_t* r1 = POLY(res, level + t, n);
    for (uint32_t i = 0; i < n; i++) {
      r0[i] = addmod(a0[(size_t)t * n + i], k0[(size_t)t * n + i], q);
      r1[i] = addmod(a1[(size_t)t * n + i], k1[(size_t)t * n + i], q);
    }
    for (int s = 0; s < ns; s++) {
      automorph_eval(c, POLY(a0, t, n), z, ks[s]);
      for (uint32_t i = 0; i < n; i++) r0[i] = addmod(r0[i], z[i], q);
    }
  }
  memcpy(out, res, sizeof(uint64_t) * 2 * (size_t)level * n);
  free(dc); free(acc); free(z); free(k0); free(k1); free(res);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Encrypted logistic-regression gradient step (Sec. 4, Eq. 5-8, Table 2).   */
/* ------------------------------------------------------------------------ */

/* Packing (after the block packing idea of Sec. 3): each data ciphertext
 * holds g samples interleaved: slot g*f + s = y_s * x_{s,f} for feature f < F
 * = (N/2)/g.  W holds w_f in slots g*f + s for every s.  The step computes
 *   w' = w + sum_k sum_s p(m_s) * z_s,  m_s = w . z_s = y_s w . x_s,
 * with p(x) = lr * (c0 + c1 x + c2 x^2 + c3 x^3) (Eq. 7-8 with the Table 2
 * polynomial, read as an ascent on the negated loss derivative), replicated
 * in all g slots of every feature.
 *
 * Op sequence and scale plan (all scales IEEE doubles, computed in this exact
 * order on both implementations; l0 = input level; q[i] the limb primes):
 *   U  = HMult(Z_k, W)                 level l0-1, sU = sZ*sW/q[l0-1]
 *   M  = sum over o < F of rot(U, o*g)   (rotsum: hoisted stages)
 *   T  = HMult(M, M)                   level l0-2, sT = sU*sU/q[l0-2]
 *   sS = ((sW*q[l0-5])*q[l0-4]) / (maskscale*sZ)         (target scale of S)
 *   sA = (sS*q[l0-3])/sT ;  A = rescale(M * round(c3*lr * sA*q[l0-2]/sU))
 *        with the constant's scale sigA = (sA*q[l0-2])/sU and A's scale
 *        (sU*sigA)/q[l0-2]
 *   C  = HMult(T, A)                   level l0-3
 *   B  = rescale(M * round(c1*lr * sigB)), sigB = (sS*q[l0-2])/sU, dropped to l0-3
 *   Q  = rescale(T * round(c2*lr * sigQ)), sigQ = (sS*q[l0-3])/sT  (if c2 != 0)
 *   S  = C + B (+ Q) + round(c0*lr * scale(C))
 *   D  = sum_k tensor(S_k, drop(Z_k, l0-3))   three parts, level l0-3
 *   G  = rescale(relinearise(D))       level l0-4, sG = scale(C)*sZ/q[l0-4]
 *        (one relinearisation and one rescale for all k: both are linear,
 *        so this encrypts sum_k S_k Z_k as the sum of nZ HMults would, with
 *        1/nZ of their key switches and less noise)
 *   H  = sum over o < g of rot(G, o)     (rotsum)
 *   H' = rescale(H (x) mask), mask = 1 on slots = 0 mod g, encoded at maskscale
 *   R  = sum over o < g of rot(H', -o)   (rotsum)
 *   W' = drop(W, l0-5) + R             level l0-5
 * Additions require scales equal to within a relative 2^-40.
 */

typedef struct { uint64_t* d; int level; double scale; } orc_ct;

static orc_ct ct_new(orc_ctx* c, int level, double scale) {
  orc_ct x; x.level = level; x.scale = scale;
  x.d = malloc(sizeof(uint64_t) * 2 * (size_t)level * c->n);
  return x;
}

static int scales_match(double a, double b) { return fabs(a / b - 1.0) < ldexp(1.0, -40); }

static int64_t round_const(double v) { return (int64_t)llround(v); }

/* x <- sum over o = 0 .. 2^count - 1 of rot(x, o * step), in hoisted stages
 * (orc_rotate_sum) of k doublings each -- rotations by s, 2s, ..., (2^k - 1) s,
 * then s <- 2^k s -- with k = 3, except k = 4 for the first stage when
 * count = 1 mod 3 (k = 1 when count = 1) and k = 2 for a last stage when
 * count = 2 mod 3. */
static int rotsum(orc_ctx* c, orc_ct* x, int32_t step, int count) {
  int sizes[32], ns = 0;
  for (int i = 0; i < count / 3; i++) sizes[ns++] = 3;
  if (count % 3 == 1) {
    if (ns == 0) sizes[ns++] = 1;
    else sizes[0] = 4;
  } else if (count % 3 == 2) {
    sizes[ns++] = 2;
  }
  int32_t s = step;
  int rc = 0;
  for (int i = 0; i < ns && rc == 0; i++) {
    int32_t st[15];
    int nr = (1 << sizes[i]) - 1;
    for (int m = 1; m <= nr; m++) st[m - 1] = s * m;
    rc = orc_rotate_sum(c, x->d, x->level, st, nr, x->d);
    s *= 1 << sizes[i];
  }
  return rc;
}

static int ilog2i(int v) { int r = 0; while ((1 << r) < v) r++; return r; }

/* Mask plaintext: 1 on slots = 0 mod g, 0 elsewhere, at scale ms. */
int orc_lr_mask(orc_ctx* c, int g, double ms, int64_t* out) {
  int nh = c->n / 2;
  double* re = calloc(nh, sizeof(double));
  for (int j = 0; j < nh; j += g) re[j] = 1.0;
  int rc = orc_encode(c, re, NULL, nh, ms, out);
  free(re);
  return rc;
}

/* The worker's update of Eq. 5-8 with a Table 2 polynomial p and, for
 * l2 > 0, the gradient of the smooth regulariser R(w) = (l2/2) |w|^2 of
 * Eq. 4 (Eq. 6 and 8: grad f = sum_i y_i grad L x_i + grad R, grad R = l2 w):
 *   w' = w + lr * (sum_i p(y_i w.x_i) y_i x_i - l2 w)
 * (the sign reading of the Table 2 polynomials and lr = eta/n as above).
 * The regulariser's term is the constant product of w taken at level l0-4,
 * by round(-lr l2 q_{l0-5}) at scale q_{l0-5}, rescaled to level l0-5 and W's
 * scale, and added last. */
int orc_lr_gradient_step(orc_ctx* c, const uint64_t* const* Z, int nZ, int levelZ, double sZ,
                         const uint64_t* Wd, int levelW, double sW, const double coeffs[4],
                         double lr, int g, double mask_scale, double l2, uint64_t* Wout, int* level_out,
                         double* scale_out) {
  uint32_t n = c->n;
  int l0 = levelZ;
  if (levelW != levelZ || l0 < 6 || nZ < 1) return -1;
  if (g < 1 || (g & (g - 1)) || g > (int)n / 2) return -1;
  int F = (int)(n / 2) / g;
  int logF = ilog2i(F), logg = ilog2i(g);
  const uint64_t* q = c->q;
  double sU = sZ * sW / (double)q[l0 - 1];
  double sT = sU * sU / (double)q[l0 - 2];
  double sS = ((sW * (double)q[l0 - 5]) * (double)q[l0 - 4]) / (mask_scale * sZ);
  double sA = (sS * (double)q[l0 - 3]) / sT;
  double sigA = (sA * (double)q[l0 - 2]) / sU;
  double sigB = (sS * (double)q[l0 - 2]) / sU;
  double sigQ = (sS * (double)q[l0 - 3]) / sT;
  int64_t kA = round_const(coeffs[3] * lr * sigA);
  int64_t kB = round_const(coeffs[1] * lr * sigB);
  int64_t kQ = round_const(coeffs[2] * lr * sigQ);
  int rc = 0;
  orc_ct G = ct_new(c, l0 - 4, 0.0);
  memset(G.d, 0, sizeof(uint64_t) * 2 * (size_t)G.level * n);
  uint64_t* tmp = malloc(sizeof(uint64_t) * 2 * (size_t)l0 * n);
  const size_t w3 = 3 * (size_t)(l0 - 3) * n;
  uint64_t* D = calloc(w3, sizeof(uint64_t));  /* sum_k tensor(S_k, Z_k) */
  double sD = 0.0;
  int have_sD = 0;
  /* the data ciphertexts' circuits are independent up to the sum D (exact
     modular addition, so its order does not matter) */
#pragma omp parallel if (nZ >= 4)
  {
    orc_ct U = ct_new(c, l0 - 1, sU), T = ct_new(c, l0 - 2, sT), A = ct_new(c, l0 - 2, 0.0);
    orc_ct Cc = ct_new(c, l0 - 3, 0.0), B = ct_new(c, l0 - 2, 0.0), Qq = ct_new(c, l0 - 3, 0.0);
    orc_ct Zd = ct_new(c, l0 - 3, sZ);
    uint64_t* tk = malloc(sizeof(uint64_t) * 2 * (size_t)l0 * n);
    uint64_t* Dk = malloc(sizeof(uint64_t) * w3);
#pragma omp for schedule(dynamic)
    for (int k = 0; k < nZ; k++) {
      int lrc = 0;
      /* U = HMult(Z_k, W); M = rotate-and-sum over the F features */
      orc_mul_relin_rescale(c, Z[k], Wd, l0, U.d);
      U.scale = sU;
      lrc = rotsum(c, &U, g, logF);
      if (lrc == 0) {
        /* T = M^2 */
        orc_mul_relin_rescale(c, U.d, U.d, l0 - 1, T.d);
        /* A = c3 * M */
        orc_mul_int(c, U.d, l0 - 1, kA, tk);
        orc_rescale(c, tk, l0 - 1, A.d);
        A.scale = (sU * sigA) / (double)q[l0 - 2];
        /* C = T * A */
        orc_mul_relin_rescale(c, T.d, A.d, l0 - 2, Cc.d);
        Cc.scale = sT * A.scale / (double)q[l0 - 3];
        /* B = c1 * M, dropped to level l0-3 */
        orc_mul_int(c, U.d, l0 - 1, kB, tk);
        orc_rescale(c, tk, l0 - 1, B.d);
        B.scale = (sU * sigB) / (double)q[l0 - 2];
        orc_drop(c, B.d, l0 - 2, l0 - 3, B.d);
        if (!scales_match(Cc.scale, B.scale)) lrc = -3;
      }
      if (lrc == 0) {
        orc_add(c, Cc.d, B.d, l0 - 3, Cc.d);
        if (coeffs[2] != 0.0) {
          orc_mul_int(c, T.d, l0 - 2, kQ, tk);
          orc_rescale(c, tk, l0 - 2, Qq.d);
          Qq.scale = (sT * sigQ) / (double)q[l0 - 3];
          if (!scales_match(Cc.scale, Qq.scale)) lrc = -3;
          else orc_add(c, Cc.d, Qq.d, l0 - 3, Cc.d);
        }
      }
      if (lrc == 0) {
        orc_add_int(c, Cc.d, l0 - 3, round_const(coeffs[0] * lr * Cc.scale), Cc.d);
        /* D += tensor(S_k, Z_k) */
        orc_drop(c, Z[k], l0, l0 - 3, Zd.d);
        orc_tensor(c, Cc.d, Zd.d, l0 - 3, Dk);
      }
#pragma omp critical(orc_lr_gradient_sum)
      {
        if (lrc) {
          rc = lrc;
        } else {
          if (!have_sD) {
            sD = Cc.scale * sZ;
            have_sD = 1;
          } else if (!scales_match(sD, Cc.scale * sZ)) {
            rc = -3;
          }
          for (int pt = 0; pt < 3; pt++)
            for (int t = 0; t < l0 - 3; t++) {
              uint64_t* dst = POLY(D, pt * (l0 - 3) + t, n);
              const uint64_t* src = POLY(Dk, pt * (l0 - 3) + t, n);
              for (uint32_t i = 0; i < n; i++) dst[i] = addmod(dst[i], src[i], q[t]);
            }
        }
      }
    }
    free(U.d); free(T.d); free(A.d); free(Cc.d); free(B.d); free(Qq.d); free(Zd.d);
    free(tk); free(Dk);
  }
  if (rc == 0) {
    /* G = rescale(relinearise(D)) */
    relin_rescale(c, D, l0 - 3, G.d);
    G.scale = sD / (double)q[l0 - 4];
    /* H = sum over the g samples of each feature (lands on slots = 0 mod g) */
    rc = rotsum(c, &G, 1, logg);
  }
  orc_ct R = ct_new(c, l0 - 5, 0.0);
  if (rc == 0) {
    int64_t* mask = malloc(sizeof(int64_t) * n);
    orc_lr_mask(c, g, mask_scale, mask);
    orc_mul_plain(c, G.d, l0 - 4, mask, tmp);
    orc_rescale(c, tmp, l0 - 4, R.d);
    R.scale = (G.scale * mask_scale) / (double)q[l0 - 5];
    free(mask);
    rc = rotsum(c, &R, -1, logg);
  }
  if (rc == 0) {
    if (!scales_match(R.scale, sW)) rc = -3;
  }
  if (rc == 0) {
    orc_drop(c, Wd, l0, l0 - 5, tmp);
    orc_add(c, tmp, R.d, l0 - 5, Wout);
    *level_out = l0 - 5;
    *scale_out = sW;
  }
  if (rc == 0 && l2 != 0.0) {
    /* - lr l2 w: w at level l0-4 times round(-lr l2 q_{l0-5}), rescaled */
    if (!(l2 > 0.0)) {
      rc = -1;
    } else {
      uint64_t* wr = malloc(sizeof(uint64_t) * 2 * (size_t)(l0 - 4) * n);
      orc_drop(c, Wd, l0, l0 - 4, wr);
      orc_mul_int(c, wr, l0 - 4, round_const(-lr * l2 * (double)q[l0 - 5]), tmp);
      orc_rescale(c, tmp, l0 - 4, wr);
      if (!scales_match((sW * (double)q[l0 - 5]) / (double)q[l0 - 5], sW)) rc = -3;
      else orc_add(c, Wout, wr, l0 - 5, Wout);
      free(wr);
    }
  }
  free(tmp);
  free(G.d); free(D); free(R.d);
  return rc;
}

/* Encrypted inference of the same model (the first half of the step): for
 * each data ciphertext, S = p(M) with M the replicated per-sample inner
 * products, following the step's op sequence up to S, with the polynomial's
 * result produced at W's scale: sS = sW (then sA, sigA, sigB, sigQ and the
 * constants as in the step).  Output: nZ ciphertexts at level l0 - 3, each
 * [2][l0-3][N] in `outs` back to back; *scale_out = the scale of S. */
int orc_lr_inference(orc_ctx* c, const uint64_t* const* Z, int nZ, int levelZ, double sZ, const uint64_t* Wd,
                     int levelW, double sW, const double coeffs[4], double lr, int g, uint64_t* outs,
                     double* scale_out) {
  uint32_t n = c->n;
  int l0 = levelZ;
  if (levelW != levelZ || l0 < 5 || nZ < 1) return -1;
  if (g < 1 || (g & (g - 1)) || g > (int)n / 2) return -1;
  int F = (int)(n / 2) / g;
  int logF = ilog2i(F);
  const uint64_t* q = c->q;
  double sU = sZ * sW / (double)q[l0 - 1];
  double sT = sU * sU / (double)q[l0 - 2];
  double sS = sW;
  double sA = (sS * (double)q[l0 - 3]) / sT;
  double sigA = (sA * (double)q[l0 - 2]) / sU;
  double sigB = (sS * (double)q[l0 - 2]) / sU;
  double sigQ = (sS * (double)q[l0 - 3]) / sT;
  int64_t kA = round_const(coeffs[3] * lr * sigA);
  int64_t kB = round_const(coeffs[1] * lr * sigB);
  int64_t kQ = round_const(coeffs[2] * lr * sigQ);
  int rc = 0;
  orc_ct U = ct_new(c, l0 - 1, sU), T = ct_new(c, l0 - 2, sT), A = ct_new(c, l0 - 2, 0.0);
  orc_ct Cc = ct_new(c, l0 - 3, 0.0), B = ct_new(c, l0 - 2, 0.0), Qq = ct_new(c, l0 - 3, 0.0);
  uint64_t* tmp = malloc(sizeof(uint64_t) * 2 * (size_t)l0 * n);
  for (int k = 0; k < nZ && rc == 0; k++) {
    orc_mul_relin_rescale(c, Z[k], Wd, l0, U.d);
    rc = rotsum(c, &U, g, logF);
    if (rc) break;
    orc_mul_relin_rescale(c, U.d, U.d, l0 - 1, T.d);
    orc_mul_int(c, U.d, l0 - 1, kA, tmp);
    orc_rescale(c, tmp, l0 - 1, A.d);
    A.scale = (sU * sigA) / (double)q[l0 - 2];
    orc_mul_relin_rescale(c, T.d, A.d, l0 - 2, Cc.d);
    Cc.scale = sT * A.scale / (double)q[l0 - 3];
    orc_mul_int(c, U.d, l0 - 1, kB, tmp);
    orc_rescale(c, tmp, l0 - 1, B.d);
    B.scale = (sU * sigB) / (double)q[l0 - 2];
    orc_drop(c, B.d, l0 - 2, l0 - 3, B.d);
    if (!scales_match(Cc.scale, B.scale)) { rc = -3; break; }
    orc_add(c, Cc.d, B.d, l0 - 3, Cc.d);
    if (coeffs[2] != 0.0) {
      orc_mul_int(c, T.d, l0 - 2, kQ, tmp);
      orc_rescale(c, tmp, l0 - 2, Qq.d);
      Qq.scale = (sT * sigQ) / (double)q[l0 - 3];
      if (!scales_match(Cc.scale, Qq.scale)) { rc = -3; break; }
      orc_add(c, Cc.d, Qq.d, l0 - 3, Cc.d);
    }
    orc_add_int(c, Cc.d, l0 - 3, round_const(coeffs[0] * lr * Cc.scale), Cc.d);
    memcpy(outs + (size_t)k * 2 * (l0 - 3) * n, Cc.d, sizeof(uint64_t) * 2 * (size_t)(l0 - 3) * n);
    *scale_out = Cc.scale;
  }
  free(tmp);
  free(U.d); free(T.d); free(A.d); free(Cc.d); free(B.d); free(Qq.d);
  return rc;
}
