// codec.cu -- encode/decode (Sec. 3: canonical embedding) and decryption.
//
// Slot j is the value at zeta_j = w^(e_j), w = exp(i pi / N), e_j = 5^j mod
// 2N; its conjugate sits at w^(2N - e_j).  With u(t) = (t - 1)/2 for odd t:
//  encode: coefficient i = (Delta/N) Re(w^-i * F(W)[i]), F the forward
//          (e^-) length-N DFT of W[u(e_j)] = z_j, W[u(2N - e_j)] = conj(z_j),
//          rounded half away from zero;
//  decode: z_j = (1/Delta) G(m w^i)[u(e_j)], G the e^+ length-N DFT.
// Decrypt: m = c0 + c1 s per limb, inverse NTT, Garner's mixed-radix digits,
// centered against (Q-1)/2, converted to double by Horner from the top digit.
#include <math.h>

#include <vector>

#include "he_internal.h"
#include "he_kernels.h"
#include "he_ops.h"

namespace he {

// ---- radix-2 complex FFT in double, one launch per stage ---------------------
__global__ void k_bitrev_copy(const double2* in, double2* out, int log_n) {
  const uint32_t n = 1u << log_n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    out[brev_bits(i, log_n)] = in[i];
}

// Stage with half-size h: pairs (i, i + h) in blocks of 2h, twiddle
// exp(sign * i pi * (i mod h) / h); sign -1 gives the e^- DFT, +1 the e^+ one.
__global__ void k_fft_stage(double2* a, int log_n, uint32_t h, double sign) {
  const uint32_t n = 1u << log_n;
  for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n / 2; g += gridDim.x * blockDim.x) {
    const uint32_t pos = g % h, blk = g / h;
    const uint32_t i0 = blk * 2 * h + pos, i1 = i0 + h;
    double sn, cs;
    sincospi(sign * (double)pos / (double)h, &sn, &cs);
    const double2 x = a[i0], y = a[i1];
    const double2 ty = make_double2(y.x * cs - y.y * sn, y.x * sn + y.y * cs);
    a[i0] = make_double2(x.x + ty.x, x.y + ty.y);
    a[i1] = make_double2(x.x - ty.x, x.y - ty.y);
  }
}

// out = DFT(in) with kernel exp(sign * 2 pi i jk / n), sign = +-1.
static int fft(he_ctx* c, double2* in, double2* out, double sign) {
  const int log_n = c->log_n;
  const uint32_t n = c->n;
  k_bitrev_copy<<<grid_for(n), 256, 0, c->stream>>>(in, out, log_n);
  for (uint32_t h = 1; h < n; h <<= 1)
    k_fft_stage<<<grid_for(n / 2), 256, 0, c->stream>>>(out, log_n, h, sign);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// W[u(e_j)] = z_j, W[u(2N - e_j)] = z_j (real slots), zero elsewhere.
__global__ void k_encode_scatter(const double* z, uint32_t nz, double2* W, int log_n) {
  const uint32_t n = 1u << log_n, m = 2 * n, nh = n / 2;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nh; j += gridDim.x * blockDim.x) {
    // e_j = 5^j mod 2N by square-and-multiply
    uint32_t e = 1, b = 5, x = j;
    while (x) {
      if (x & 1) e = (uint32_t)(((uint64_t)e * b) & (m - 1));
      b = (uint32_t)(((uint64_t)b * b) & (m - 1));
      x >>= 1;
    }
    const double v = j < nz ? z[j] : 0.0;
    W[(e - 1) / 2] = make_double2(v, 0.0);
    W[(m - e - 1) / 2] = make_double2(v, 0.0);
  }
}

__global__ void k_encode_finish(const double2* F, int64_t* out, double scale, int log_n, int* overflow) {
  const uint32_t n = 1u << log_n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi(-(double)i / (double)n, &sn, &cs);  // w^-i
    const double re = F[i].x * cs - F[i].y * sn;
    const double raw = (scale / (double)n) * re;
    if (!(fabs(raw) < 9.2e18)) {
      *overflow = 1;
      out[i] = 0;
    } else {
      out[i] = llround(raw);
    }
  }
}

// Encode device slots d_z (n_slots doubles) into device int64 coefficients
// d_out.  scratch: 2N double2; d_ovf: one int (set when a coefficient leaves int64).
int encode_dev(he_ctx* c, const double* d_z, size_t n_slots, double scale, int64_t* d_out,
               double2* scratch, int* d_ovf) {
  const uint32_t n = c->n;
  if (n_slots > n / 2) return fail(HE_EINVAL, "more slots than N/2");
  if (!(scale > 0.0)) return fail(HE_EINVAL, "scale must be positive");
  double2* W = scratch;
  double2* F = scratch + n;
  HE_CUDA(cudaMemsetAsync(W, 0, sizeof(double2) * n, c->stream));
  k_encode_scatter<<<grid_for(n / 2), 256, 0, c->stream>>>(d_z, (uint32_t)n_slots, W, c->log_n);
  HE_TRY(fft(c, W, F, -1.0));
  k_encode_finish<<<grid_for(n), 256, 0, c->stream>>>(F, d_out, scale, c->log_n, d_ovf);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// ---- decryption -----------------------------------------------------------------
__global__ void k_decrypt_dot(CtBatch A, const uint64_t* s, uint64_t* m, uint32_t level, int log_n,
                              const PrimeDev* primes) {
  const uint32_t n = 1u << log_n;
  const size_t total = (size_t)level * n;
  for (size_t g = blockIdx.x * (size_t)blockDim.x + threadIdx.x; g < total; g += (size_t)gridDim.x * blockDim.x) {
    const uint32_t t = (uint32_t)(g / n), k = (uint32_t)(g % n);
    const PrimeDev pr = primes[t];
    const uint64_t c0 = A.base[(size_t)t * n + k], c1 = A.base[((size_t)A.cap + t) * n + k];
    m[g] = add_mod(c0, mul_mod(c1, s[(size_t)t * n + k], pr), pr.q);
  }
}

struct GarnerArgs {
  uint64_t half[HE_MAX_PRIMES];  // mixed-radix digits of (Q-1)/2
};

// gar: [L] Shoup pairs of (q_0..q_{i-1})^-1 mod q_i, then [L][L] prefix products
// (q_0..q_{i'-1}) mod q_i at [i][i'].
__global__ void k_crt_double(const uint64_t* m, double* out, uint32_t level, int log_n,
                             const PrimeDev* primes, const uint64_t* gar, uint32_t L, GarnerArgs ga) {
  const uint32_t n = 1u << log_n;
  for (uint32_t k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
    uint64_t d[HE_MAX_PRIMES];
    for (uint32_t i = 0; i < level; ++i) {
      const PrimeDev pr = primes[i];
      const uint64_t* pref = gar + 2 * L + (size_t)i * L;
      uint64_t acc = 0;
      for (uint32_t j = 0; j < i; ++j) acc = add_mod(acc, mul_mod(reduce64(d[j], pr), pref[j], pr), pr.q);
      const uint64_t x = sub_mod(m[(size_t)i * n + k], acc, pr.q);
      d[i] = i ? mul_shoup(x, gar[2 * i], gar[2 * i + 1], pr.q) : x;
    }
    int cmp = 0;
    for (int i = (int)level - 1; i >= 0 && cmp == 0; --i)
      cmp = d[i] > ga.half[i] ? 1 : (d[i] < ga.half[i] ? -1 : 0);
    const bool neg = cmp > 0;
    if (neg) {  // Q - v = (Q - 1 - v) + 1
      uint64_t carry = 1;
      for (uint32_t i = 0; i < level; ++i) {
        uint64_t v = primes[i].q - 1 - d[i] + carry;
        carry = 0;
        if (v == primes[i].q) { v = 0; carry = 1; }
        d[i] = v;
      }
    }
    double v = (double)d[level - 1];
    for (int i = (int)level - 2; i >= 0; --i) v = v * (double)primes[i].q + (double)d[i];
    out[k] = neg ? -v : v;
  }
}

// scratch m: level*N words.
int decrypt_dev(he_ctx* c, const he_ct* ct, uint64_t* m, double* d_coeffs) {
  const uint32_t n = c->n, level = ct->level;
  const size_t lw = (size_t)level * n;
  CtBatch A{ct->data, 0, ct->cap, 0};
  k_decrypt_dot<<<grid_for(lw), 256, 0, c->stream>>>(A, c->d_s, m, level, c->log_n, c->d_primes);
  HE_CUDA(cudaGetLastError());
  PolyBatch b;
  b.src = m;
  b.dst = m;
  b.src_stride = b.dst_stride = 0;
  b.npolys = 1;
  b.nl = level;
  b.limb0 = 0;
  b.level = c->L;
  b.skip_alpha = 0;
  b.skip_beta = 1;
  HE_TRY(ntt_inverse(c, b));
  // digits of (Q-1)/2: Q-1 has digits q_i - 1; halve from the top digit down
  GarnerArgs ga;
  unsigned __int128 carry = 0;
  for (int i = (int)level - 1; i >= 0; --i) {
    const unsigned __int128 cur = carry * c->q[i] + (c->q[i] - 1);
    ga.half[i] = (uint64_t)(cur / 2);
    carry = cur % 2;
  }
  k_crt_double<<<grid_for(n), 256, 0, c->stream>>>(m, d_coeffs, level, c->log_n, c->d_primes,
                                                   c->d_garner, (uint32_t)c->L, ga);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

// W_i = m_i w^i (m as centered doubles), then G = e^+ DFT; slot j = G[u(e_j)] / scale.
__global__ void k_decode_twist(const double* m, double2* W, int log_n) {
  const uint32_t n = 1u << log_n;
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double sn, cs;
    sincospi((double)i / (double)n, &sn, &cs);
    W[i] = make_double2(m[i] * cs, m[i] * sn);
  }
}

__global__ void k_decode_gather(const double2* G, double* re, double* im, uint32_t nz, double scale,
                                int log_n) {
  const uint32_t n = 1u << log_n, m = 2 * n;
  for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < nz; j += gridDim.x * blockDim.x) {
    uint32_t e = 1, b = 5, x = j;
    while (x) {
      if (x & 1) e = (uint32_t)(((uint64_t)e * b) & (m - 1));
      b = (uint32_t)(((uint64_t)b * b) & (m - 1));
      x >>= 1;
    }
    const double2 v = G[(e - 1) / 2];
    re[j] = v.x / scale;
    if (im) im[j] = v.y / scale;
  }
}

// Decode centered coefficients (device doubles d_m) into n_slots device
// values d_re.  scratch: 2N double2.
int decode_dev(he_ctx* c, const double* d_m, double scale, double* d_re, size_t n_slots,
               double2* scratch) {
  const uint32_t n = c->n;
  if (n_slots > n / 2) return fail(HE_EINVAL, "more slots than N/2");
  double2* W = scratch;
  double2* G = scratch + n;
  k_decode_twist<<<grid_for(n), 256, 0, c->stream>>>(d_m, W, c->log_n);
  HE_TRY(fft(c, W, G, 1.0));
  k_decode_gather<<<grid_for(n_slots), 256, 0, c->stream>>>(G, d_re, nullptr, (uint32_t)n_slots, scale,
                                                            c->log_n);
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

}  // namespace he
