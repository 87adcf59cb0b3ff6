// params.cu -- host number theory and the constant tables the kernels read:
// primes, roots, NTT twiddles with Shoup companions, basis-conversion,
// ModDown and rescale constants, the Gaussian table.
//
// Conventions (free choices the paper leaves open; Sec. 3 names only N and
// the modulus size):
//  * primes: q = k*2N + 1 scanned downward from 2^bits, primes kept in the
//    order found; limbs at limb_bits, then special primes at special_bits
//    skipping any limb;
//  * psi: the least residue of multiplicative order exactly 2N;
//  * NTT order: evaluation at psi^(2*brv(j)+1) in slot j.
#include <math.h>
#include <string.h>

#include <string>
#include <vector>

#include "he_internal.h"

namespace he {

typedef unsigned __int128 u128;

uint64_t h_mulmod(uint64_t a, uint64_t b, uint64_t q) { return (uint64_t)((u128)a * b % q); }

uint64_t h_powmod(uint64_t a, uint64_t e, uint64_t q) {
  uint64_t r = 1 % q;
  a %= q;
  for (; e; e >>= 1) {
    if (e & 1) r = h_mulmod(r, a, q);
    a = h_mulmod(a, a, q);
  }
  return r;
}

uint64_t h_invmod(uint64_t a, uint64_t q) { return h_powmod(a, q - 2, q); }

uint64_t h_shoup(uint64_t w, uint64_t q) { return (uint64_t)(((u128)w << 64) / q); }

// Deterministic Miller-Rabin for 64-bit n: witnesses 2..37 suffice.
bool h_is_prime(uint64_t n) {
  const uint64_t wit[12] = {2, 3, 5, 7, 11, 13, 17, 19, 23, 29, 31, 37};
  if (n < 2) return false;
  for (uint64_t p : wit) {
    if (n % p == 0) return n == p;
  }
  uint64_t d = n - 1;
  int r = 0;
  while (!(d & 1)) {
    d >>= 1;
    ++r;
  }
  for (uint64_t a : wit) {
    uint64_t x = h_powmod(a, d, n);
    if (x == 1 || x == n - 1) continue;
    bool witness = true;
    for (int i = 1; i < r && witness; ++i) {
      x = h_mulmod(x, x, n);
      if (x == n - 1) witness = false;
    }
    if (witness) return false;
  }
  return true;
}

std::vector<uint64_t> h_ntt_primes(int bits, int log_n, int count, const std::vector<uint64_t>& skip) {
  std::vector<uint64_t> out;
  const uint64_t m = 2ull << log_n;
  const uint64_t top = (1ull << bits) - 1;
  for (uint64_t k = (top - 1) / m; k > 0 && (int)out.size() < count; --k) {
    uint64_t q = k * m + 1;
    bool used = false;
    for (uint64_t s : skip) used |= (s == q);
    if (!used && h_is_prime(q)) out.push_back(q);
  }
  return out;
}

// Least element of order 2N: every primitive 2N-th root is an odd power of
// g^((q-1)/2N) for a quadratic non-residue g; take the minimum of them.
uint64_t h_min_root(uint64_t q, int log_n) {
  const uint64_t n = 1ull << log_n;
  uint64_t g = 2;
  while (h_powmod(g, (q - 1) >> 1, q) != q - 1) ++g;
  const uint64_t r0 = h_powmod(g, (q - 1) / (2 * n), q);
  const uint64_t r2 = h_mulmod(r0, r0, q);
  uint64_t best = r0, x = r0;
  for (uint64_t i = 1; i < n; ++i) {
    x = h_mulmod(x, r2, q);
    if (x < best) best = x;
  }
  return best;
}

// Discrete Gaussian cumulative table (see the sampler in keys.cu):
// K = ceil(6 sigma); T[k] = floor(2^64 * (rho0 + 2 sum_{1..k} rho_i) / Z).
int h_gauss_table(double sigma, uint64_t* T) {
  const int K = (int)ceil(6.0 * sigma);
  if (K < 1 || K > 255) return -1;
  const double denom = 2.0 * sigma * sigma;
  std::vector<double> rho(K + 1);
  for (int k = 0; k <= K; ++k) rho[k] = exp(-((double)(k * k)) / denom);
  double z = rho[0];
  for (int k = 1; k <= K; ++k) z += 2.0 * rho[k];
  double cum = rho[0];
  T[0] = (uint64_t)ldexp(cum / z, 64);
  for (int k = 1; k < K; ++k) {
    cum += 2.0 * rho[k];
    T[k] = (uint64_t)ldexp(cum / z, 64);
  }
  return K;
}

// Galois element of a left rotation by r: 5^(r mod N/2) mod 2N.
uint64_t h_galois_elt(int log_n, int32_t r) {
  const int64_t slots = 1ll << (log_n - 1);
  int64_t e = ((int64_t)r % slots + slots) % slots;
  return h_powmod(5, (uint64_t)e, 2ull << log_n);
}

static uint32_t brv_host(uint32_t x, int bits) {
  uint32_t r = 0;
  for (int i = 0; i < bits; ++i) {
    r = (r << 1) | (x & 1);
    x >>= 1;
  }
  return r;
}

static int bitlen(uint64_t q) {
  int k = 0;
  while (k < 64 && (q >> k)) ++k;
  return k;
}

// Build every table and upload it.  Returns an HE_* code.
int build_tables(he_ctx* c) {
  const int n = c->n, np = c->np, L = c->L, alpha = c->alpha;
  // primes and roots
  c->q = h_ntt_primes((int)c->prm.limb_bits, c->log_n, L, {});
  if ((int)c->q.size() != L) return fail(HE_EINVAL, "not enough limb primes at this size");
  std::vector<uint64_t> sp = h_ntt_primes((int)c->prm.special_bits, c->log_n, alpha, c->q);
  if ((int)sp.size() != alpha) return fail(HE_EINVAL, "not enough special primes at this size");
  c->q.insert(c->q.end(), sp.begin(), sp.end());
  c->psi.resize(np);
  for (int t = 0; t < np; ++t) c->psi[t] = h_min_root(c->q[t], c->log_n);

  // primes + Barrett constants
  std::vector<PrimeDev> pd(np);
  std::vector<uint64_t> two64(np);
  for (int t = 0; t < np; ++t) {
    const uint64_t q = c->q[t];
    PrimeDev& p = pd[t];
    memset(&p, 0, sizeof p);
    p.q = q;
    p.k = (uint32_t)bitlen(q);
    p.mu = (uint64_t)(((u128)1 << (2 * p.k)) / q);
    p.n_inv = h_invmod((uint64_t)n % q, q);
    p.n_inv_sh = h_shoup(p.n_inv, q);
    p.one_sh = h_shoup(1, q);
    two64[t] = (uint64_t)(((u128)1 << 64) % q);
    p.r64 = two64[t];
    p.r64_sh = h_shoup(p.r64, q);
  }
  HE_CUDA(cudaMalloc(&c->d_primes, sizeof(PrimeDev) * np));
  HE_CUDA(cudaMemcpy(c->d_primes, pd.data(), sizeof(PrimeDev) * np, cudaMemcpyHostToDevice));
  HE_CUDA(cudaMalloc(&c->d_two64, sizeof(uint64_t) * np));
  HE_CUDA(cudaMemcpy(c->d_two64, two64.data(), sizeof(uint64_t) * np, cudaMemcpyHostToDevice));

  // twiddles: tw[m] = psi^brv(m), itw[m] = psi^-brv(m), interleaved with Shoup companions
  {
    std::vector<uint64_t> tw((size_t)np * n * 2), itw((size_t)np * n * 2), pw(n), ipw(n);
    for (int t = 0; t < np; ++t) {
      const uint64_t q = c->q[t], ps = c->psi[t], ips = h_invmod(ps, q);
      pw[0] = 1;
      ipw[0] = 1;
      for (int i = 1; i < n; ++i) {
        pw[i] = h_mulmod(pw[i - 1], ps, q);
        ipw[i] = h_mulmod(ipw[i - 1], ips, q);
      }
      for (int m = 0; m < n; ++m) {
        const uint32_t r = brv_host((uint32_t)m, c->log_n);
        size_t o = ((size_t)t * n + m) * 2;
        tw[o] = pw[r];
        tw[o + 1] = h_shoup(pw[r], q);
        itw[o] = ipw[r];
        itw[o + 1] = h_shoup(ipw[r], q);
      }
    }
    HE_CUDA(cudaMalloc(&c->d_tw, sizeof(uint64_t) * tw.size()));
    HE_CUDA(cudaMemcpy(c->d_tw, tw.data(), sizeof(uint64_t) * tw.size(), cudaMemcpyHostToDevice));
    HE_CUDA(cudaMalloc(&c->d_itw, sizeof(uint64_t) * itw.size()));
    HE_CUDA(cudaMemcpy(c->d_itw, itw.data(), sizeof(uint64_t) * itw.size(), cudaMemcpyHostToDevice));
  }

  // Gaussian table
  {
    uint64_t T[256];
    c->gK = h_gauss_table(c->prm.sigma, T);
    if (c->gK < 1) return fail(HE_EINVAL, "sigma out of range");
    HE_CUDA(cudaMalloc(&c->d_gauss, sizeof(uint64_t) * c->gK));
    HE_CUDA(cudaMemcpy(c->d_gauss, T, sizeof(uint64_t) * c->gK, cudaMemcpyHostToDevice));
  }

  // ModUp constants per (level, digit): digit D_j = [j*alpha, min((j+1)*alpha, level)).
  // Table: [cnt] Shoup pairs (inv_i = (Q_j/q_i)^-1 mod q_i), then [cnt][np] values
  // (Q_j/q_i) mod p for every prime index p, then their [cnt][np] Shoup companions,
  // then [cnt] Shoup pairs of inv_i * N^-1 mod q_i (the conversion's first product
  // folded with the scaling that ends an inverse transform).
  {
    std::vector<uint64_t> words;
    c->modup.assign(L + 1, {});
    for (int lv = 1; lv <= L; ++lv) {
      const int beta_l = (lv + alpha - 1) / alpha;
      for (int j = 0; j < beta_l; ++j) {
        ModUpConst mc;
        mc.lo = (uint32_t)(j * alpha);
        mc.cnt = (uint32_t)(std::min((j + 1) * alpha, lv) - j * alpha);
        mc.off = words.size();
        for (uint32_t a = 0; a < mc.cnt; ++a) {
          const int i = (int)(mc.lo + a);
          uint64_t qi = c->q[i], prod = 1 % qi;
          for (uint32_t b = 0; b < mc.cnt; ++b)
            if (b != a) prod = h_mulmod(prod, c->q[mc.lo + b] % qi, qi);
          const uint64_t inv = h_invmod(prod, qi);
          words.push_back(inv);
          words.push_back(h_shoup(inv, qi));
        }
        const size_t mat0 = words.size();
        for (uint32_t a = 0; a < mc.cnt; ++a) {
          for (int p = 0; p < np; ++p) {
            const uint64_t m = c->q[p];
            uint64_t prod = 1 % m;
            for (uint32_t b = 0; b < mc.cnt; ++b)
              if (b != a) prod = h_mulmod(prod, c->q[mc.lo + b] % m, m);
            words.push_back(prod);
          }
        }
        for (uint32_t a = 0; a < mc.cnt; ++a)
          for (int p = 0; p < np; ++p) words.push_back(h_shoup(words[mat0 + (size_t)a * np + p], c->q[p]));
        for (uint32_t a = 0; a < mc.cnt; ++a) {
          const uint64_t qi = c->q[mc.lo + a];
          const uint64_t v = h_mulmod(words[mc.off + 2 * a], h_invmod((uint64_t)n % qi, qi), qi);
          words.push_back(v);
          words.push_back(h_shoup(v, qi));
        }
        c->modup[lv].push_back(mc);
      }
    }
    HE_CUDA(cudaMalloc(&c->d_modup, sizeof(uint64_t) * words.size()));
    HE_CUDA(cudaMemcpy(c->d_modup, words.data(), sizeof(uint64_t) * words.size(), cudaMemcpyHostToDevice));
  }

  // ModDown constants for dividing by the product P of the dropped primes
  // drop[0 .. a) (the special primes; with q_{l-1} first, the ModDown merged
  // with a rescale): [a] Shoup pairs of (P/p_k)^-1 mod p_k; [a][L] values
  // (P/p_k) mod q_t; [L] Shoup pairs of P^-1 mod q_t; then h = (P-1)/2
  // reduced: [a] h mod p_k and [L] h mod q_t (the division by P rounds); then
  // the [a][L] Shoup companions of the (P/p_k) mod q_t values; [a] low words
  // of floor(2^128 / p_k) (the high word is floor(2^64 / p_k)); [L] P mod q_t;
  // [L][8] v P mod q_t.  The last two make the conversion exact: v =
  // floor(sum_k u_k / p_k) is evaluated in 64.64 fixed point and v P
  // subtracted.  Then, for the rare elements whose fixed-point sum lies
  // within its error of an integer, the integers themselves: [a][8] words of
  // P/p_k and [8] words of P (little-endian 64-bit words; a <= 8 primes below
  // 2^61 keep sum_k u_k P/p_k and 8 P below 2^512).  4a + 2aL + 12L + 8a + 8
  // words.
  auto md_words = [&](const std::vector<int>& drop) {
    const int a = (int)drop.size();
    std::vector<uint64_t> words;
    auto prod_mod = [&](uint64_t m, int skip) {  // prod of drop[] except drop[skip], mod m
      uint64_t r = 1 % m;
      for (int k2 = 0; k2 < a; ++k2)
        if (k2 != skip) r = h_mulmod(r, c->q[drop[k2]] % m, m);
      return r;
    };
    for (int k = 0; k < a; ++k) {
      const uint64_t pk = c->q[drop[k]];
      const uint64_t inv = h_invmod(prod_mod(pk, k), pk);
      words.push_back(inv);
      words.push_back(h_shoup(inv, pk));
    }
    for (int k = 0; k < a; ++k)
      for (int t = 0; t < L; ++t) words.push_back(prod_mod(c->q[t], k));
    std::vector<uint64_t> Pq(L);
    for (int t = 0; t < L; ++t) {
      const uint64_t qt = c->q[t];
      Pq[t] = prod_mod(qt, -1);
      const uint64_t inv = Pq[t] ? h_invmod(Pq[t], qt) : 0;  // P = 0 mod q_t only for a dropped q_t (not a target)
      words.push_back(inv);
      words.push_back(h_shoup(inv, qt));
    }
    auto half_P = [&](uint64_t m) {  // (P - 1)/2 mod m = (P mod m - 1) * 2^-1 mod m
      return h_mulmod((prod_mod(m, -1) + m - 1) % m, h_invmod(2, m), m);
    };
    for (int k = 0; k < a; ++k) words.push_back(half_P(c->q[drop[k]]));
    for (int t = 0; t < L; ++t) words.push_back(half_P(c->q[t]));
    for (int k = 0; k < a; ++k)
      for (int t = 0; t < L; ++t) words.push_back(h_shoup(words[2 * a + (size_t)k * L + t], c->q[t]));
    for (int k = 0; k < a; ++k) words.push_back((uint64_t)(~(unsigned __int128)0 / c->q[drop[k]]));
    for (int t = 0; t < L; ++t) words.push_back(Pq[t]);
    for (int t = 0; t < L; ++t)  // [L][8]: v P mod q_t for v = 0 .. 7 (v < a <= 8)
      for (uint64_t v = 0; v < 8; ++v) words.push_back(h_mulmod(v % c->q[t], Pq[t], c->q[t]));
    auto prod_words = [&](int skip) {  // prod of drop[] except drop[skip], as 8 words
      std::vector<uint64_t> x(8, 0);
      x[0] = 1;
      for (int k2 = 0; k2 < a; ++k2) {
        if (k2 == skip) continue;
        u128 carry = 0;
        for (int w = 0; w < 8; ++w) {
          const u128 t = (u128)x[w] * c->q[drop[k2]] + carry;
          x[w] = (uint64_t)t;
          carry = t >> 64;
        }
      }
      return x;
    };
    for (int k = 0; k < a; ++k)
      for (uint64_t w : prod_words(k)) words.push_back(w);
    for (uint64_t w : prod_words(-1)) words.push_back(w);
    return words;
  };
  {
    std::vector<int> sp;
    for (int k = 0; k < alpha; ++k) sp.push_back(L + k);
    const std::vector<uint64_t> words = md_words(sp);
    c->P_mod_q.assign(L, 0);
    const size_t pq_off = 4 * (size_t)alpha + 2 * (size_t)alpha * L + 3 * (size_t)L;  // the [L] P mod q_t
    for (int t = 0; t < L; ++t) c->P_mod_q[t] = words[pq_off + t];
    HE_CUDA(cudaMalloc(&c->d_moddown, sizeof(uint64_t) * words.size()));
    HE_CUDA(cudaMemcpy(c->d_moddown, words.data(), sizeof(uint64_t) * words.size(), cudaMemcpyHostToDevice));
  }
  // The same for dividing by P q_{l-1} (ModDown merged with the rescale of a
  // multiplication at level l, 2 <= l <= L): dropped primes q_{l-1}, then the
  // special primes; one table of 12(alpha+1) + 2(alpha+1)L + 12L + 8 words per l.
  if (alpha + 1 <= 8) {
    const size_t W = 12 * (size_t)(alpha + 1) + 2 * (size_t)(alpha + 1) * L + 12 * (size_t)L + 8;
    std::vector<uint64_t> all(W * (L + 1), 0);
    for (int l = 2; l <= L; ++l) {
      std::vector<int> drop{l - 1};
      for (int k = 0; k < alpha; ++k) drop.push_back(L + k);
      const std::vector<uint64_t> words = md_words(drop);
      std::copy(words.begin(), words.end(), all.begin() + W * l);
    }
    c->mdrs_words = W;
    HE_CUDA(cudaMalloc(&c->d_mdrs, sizeof(uint64_t) * all.size()));
    HE_CUDA(cudaMemcpy(c->d_mdrs, all.data(), sizeof(uint64_t) * all.size(), cudaMemcpyHostToDevice));
  }

  // Rescale constants: for dropping limb l (1 <= l < L), q_l^-1 mod q_t for t < l.
  {
    std::vector<uint64_t> words((size_t)L * L * 2, 0);
    for (int l = 1; l < L; ++l)
      for (int t = 0; t < l; ++t) {
        const uint64_t inv = h_invmod(c->q[l] % c->q[t], c->q[t]);
        size_t o = ((size_t)l * L + t) * 2;
        words[o] = inv;
        words[o + 1] = h_shoup(inv, c->q[t]);
      }
    HE_CUDA(cudaMalloc(&c->d_rescale, sizeof(uint64_t) * words.size()));
    HE_CUDA(cudaMemcpy(c->d_rescale, words.data(), sizeof(uint64_t) * words.size(), cudaMemcpyHostToDevice));
  }
  // The rescale is a ModDown by the single prime q_l (rounded the same way):
  // per l, the ModDown table layout with alpha = 1 and q_l as the special
  // prime (Shoup pairs of 1; [L] 1; [L] Shoup pairs of q_l^-1 mod q_t; h =
  // (q_l - 1)/2 and [L] h mod q_t; [L] Shoup companions of 1; an unused word;
  // [L] q_l mod q_t; [L][8] v q_l mod q_t), for the fused kernels.
  {
    const size_t W = 4 + 14 * (size_t)L;
    std::vector<uint64_t> words(W * L, 0);
    for (int l = 1; l < L; ++l) {
      uint64_t* b = words.data() + (size_t)l * W;
      const uint64_t ql = c->q[l], h = (ql - 1) / 2;
      b[0] = 1;
      b[1] = h_shoup(1, ql);
      for (int t = 0; t < L; ++t) {
        const uint64_t qt = c->q[t];
        b[2 + t] = 1 % qt;
        if (t < l) {
          const uint64_t inv = h_invmod(ql % qt, qt);
          b[2 + L + 2 * t] = inv;
          b[2 + L + 2 * t + 1] = h_shoup(inv, qt);
        }
        b[3 + 3 * L + t] = h % qt;
        b[3 + 4 * L + t] = h_shoup(1 % qt, qt);
        b[4 + 5 * L + t] = ql % qt;
        for (uint64_t v = 0; v < 8; ++v) b[4 + 6 * L + (size_t)t * 8 + v] = h_mulmod(v % qt, ql % qt, qt);
      }
      b[2 + 3 * L] = h;
    }
    c->rescale_md_words = W;
    HE_CUDA(cudaMalloc(&c->d_rescale_md, sizeof(uint64_t) * words.size()));
    HE_CUDA(cudaMemcpy(c->d_rescale_md, words.data(), sizeof(uint64_t) * words.size(), cudaMemcpyHostToDevice));
  }
  // Garner constants for decryption
  {
    std::vector<uint64_t> words((size_t)L * 2 + (size_t)L * L, 0);
    for (int i = 0; i < L; ++i) {
      const uint64_t qi = c->q[i];
      uint64_t pref = 1 % qi;
      for (int j = 0; j < L; ++j) {
        words[(size_t)L * 2 + (size_t)i * L + j] = pref;  // (q_0..q_{j-1}) mod q_i
        pref = h_mulmod(pref, c->q[j] % qi, qi);
      }
      uint64_t prod = 1 % qi;
      for (int j = 0; j < i; ++j) prod = h_mulmod(prod, c->q[j] % qi, qi);
      const uint64_t inv = i ? h_invmod(prod, qi) : 1;
      words[2 * i] = inv;
      words[2 * i + 1] = h_shoup(inv, qi);
    }
    HE_CUDA(cudaMalloc(&c->d_garner, sizeof(uint64_t) * words.size()));
    HE_CUDA(cudaMemcpy(c->d_garner, words.data(), sizeof(uint64_t) * words.size(), cudaMemcpyHostToDevice));
  }
  // copies from pageable memory may still be in flight when cudaMemcpy
  // returns; kernels on a non-blocking stream would not wait for them
  HE_CUDA(cudaDeviceSynchronize());
  return HE_OK;
}

}  // namespace he
