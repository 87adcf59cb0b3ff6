// ntt.cu -- negacyclic number-theoretic transforms over batches of limbs.
//
// Forward transform (natural order in, bit-reversed evaluation order out):
// Cooley-Tukey stages s = 0..n-1; stage s pairs i and i + N/2^(s+1) (bit
// n-1-s of i clear) with twiddle tw[2^s + (i >> (n-s))], tw[m] = psi^brv(m).
// Inverse: Gentleman-Sande stages s = n-1..0 with psi^-brv(m), then N^-1.
// The transform evaluates at psi^(2*brv(j)+1) in slot j -- the residue layout
// every kernel and the ABI use.
//
// Launch shape: for N >= 2^12 two passes; the first covers the top n1 index
// bits ("column" transforms, elements 2^(n-n1) apart), the second the low
// n - n1 bits (contiguous "row" transforms).  A CTA loads a tile of K
// transforms into shared memory with coalesced loads, runs radix-8 rounds
// (three stages per round, eight residues in registers per thread), and
// writes the tile back.  Butterflies are Harvey's lazy ones (forward values
// in [0, 4q), inverse in [0, 2q), Shoup products); the last pass returns
// canonical residues.
#include <algorithm>

#include "he_internal.h"

namespace he {

struct NttPassArgs {
  const uint64_t* src;
  uint64_t* dst;
  uint64_t src_stride, dst_stride;
  uint32_t nl, limb0, level, L;
  uint32_t skip_alpha, skip_beta;
  const ulonglong2* tw;  // twiddle pairs (value, Shoup companion), [np][N]
  const PrimeDev* primes;
  int log_n, log_m, bit_lo, K, log_k, tiles_per_limb;
  int last;  // final pass: canonical output (and N^-1 for the inverse)
};

template <bool COL>
__device__ __forceinline__ uint32_t elem_index(const NttPassArgs& a, uint32_t tile, uint32_t k, uint32_t x) {
  const uint32_t f = tile * (uint32_t)a.K + k;
  return COL ? ((x << a.bit_lo) | f) : ((f << a.log_m) | x);
}

// Shared-memory slot of tile element (k, x), padded by one word per eight so
// that the stride-8 accesses of the last forward round do not share banks.
__device__ __forceinline__ uint32_t pad8(uint32_t i) { return i + (i >> 3); }

template <bool COL>
__device__ __forceinline__ uint32_t smem_index(const NttPassArgs& a, uint32_t k, uint32_t x) {
  return pad8(COL ? ((x << a.log_k) | k) : ((k << a.log_m) | x));
}

// One round of R stages on every group of 2^R residues.
template <bool INV, bool COL, int R>
__device__ __forceinline__ void ntt_round(const NttPassArgs& a, uint64_t* sm, uint32_t tile, int sig0,
                                          const ulonglong2* tw, uint64_t q) {
  constexpr int G = 1 << R;       // residues per group
  constexpr int GPT = 8 >> R;     // groups per thread
  const uint64_t q2 = q + q;
  const int lo_bits = a.log_m - sig0 - R;
  const uint32_t lo_mask = (1u << lo_bits) - 1;
  const int stage0 = a.log_n - a.bit_lo - a.log_m + sig0;  // global stage of local stage sig0
  const uint32_t T = blockDim.x;
#pragma unroll
  for (int u = 0; u < GPT; ++u) {
    const uint32_t g = threadIdx.x + u * T;
    uint32_t k, xhi, xlo;
    if (COL) {
      k = g & (a.K - 1);
      const uint32_t r = g >> a.log_k;
      xlo = r & lo_mask;
      xhi = r >> lo_bits;
    } else {
      xlo = g & lo_mask;
      const uint32_t r = g >> lo_bits;
      xhi = r & ((1u << sig0) - 1);
      k = r >> sig0;
    }
    const uint32_t xbase = (xhi << (a.log_m - sig0)) | xlo;
    uint64_t v[G];
    uint32_t si[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
      const uint32_t x = xbase | ((uint32_t)j << lo_bits);
      si[j] = smem_index<COL>(a, k, x);
      v[j] = sm[si[j]];
    }
    const uint32_t i0 = elem_index<COL>(a, tile, k, xbase);
    if (!INV) {
#pragma unroll
      for (int st = 0; st < R; ++st) {
        const int s = stage0 + st;
        const int half = G >> (st + 1);
#pragma unroll
        for (int j = 0; j < G; ++j) {
          if (j & half) continue;
          const uint32_t i = i0 | ((uint32_t)j << (lo_bits + a.bit_lo));
          const ulonglong2 w = tw[(1u << s) + (i >> (a.log_n - s))];
          uint64_t X = v[j];
          X = X >= q2 ? X - q2 : X;
          const uint64_t t = mul_shoup_lazy(v[j + half], w.x, w.y, q);
          v[j] = X + t;
          v[j + half] = X + q2 - t;
        }
      }
    } else {
#pragma unroll
      for (int st = R - 1; st >= 0; --st) {
        const int s = stage0 + st;
        const int half = G >> (st + 1);
#pragma unroll
        for (int j = 0; j < G; ++j) {
          if (j & half) continue;
          const uint32_t i = i0 | ((uint32_t)j << (lo_bits + a.bit_lo));
          const ulonglong2 w = tw[(1u << s) + (i >> (a.log_n - s))];
          const uint64_t X = v[j], Y = v[j + half];
          uint64_t sum = X + Y;
          sum = sum >= q2 ? sum - q2 : sum;
          v[j + half] = mul_shoup_lazy(X + q2 - Y, w.x, w.y, q);
          v[j] = sum;
        }
      }
    }
#pragma unroll
    for (int j = 0; j < G; ++j) sm[si[j]] = v[j];
  }
}

template <bool INV, bool COL>
__global__ void __launch_bounds__(512) ntt_pass_kernel(NttPassArgs a) {
  extern __shared__ uint64_t sm[];
  const uint32_t n = 1u << a.log_n;
  const uint32_t M = 1u << a.log_m;
  const uint32_t tilesz = M << a.log_k;
  const uint32_t lt = blockIdx.x / a.tiles_per_limb;
  const uint32_t tile = blockIdx.x - lt * a.tiles_per_limb;
  const uint32_t p = lt / a.nl, t = a.limb0 + (lt - p * a.nl);
  if (a.skip_alpha) {
    const uint32_t j = p % a.skip_beta, lo = j * a.skip_alpha;
    const uint32_t hi = min(lo + a.skip_alpha, a.level);
    if (t >= lo && t < hi) return;
  }
  const uint32_t prime = t < a.level ? t : a.L + t - a.level;
  const PrimeDev pr = a.primes[prime];
  const uint64_t q = pr.q, q2 = q + q;
  const uint64_t* src = a.src + p * a.src_stride + (size_t)(t - a.limb0) * n;
  uint64_t* dst = a.dst + p * a.dst_stride + (size_t)(t - a.limb0) * n;
  const ulonglong2* tw = a.tw + (size_t)prime * n;

  for (uint32_t idx = threadIdx.x; idx < tilesz; idx += blockDim.x) {
    uint32_t k, x;
    if (COL) { x = idx >> a.log_k; k = idx & (a.K - 1); }
    else { k = idx >> a.log_m; x = idx & (M - 1); }
    sm[pad8(idx)] = __ldg(src + elem_index<COL>(a, tile, k, x));
  }
  __syncthreads();

  const int nr = (a.log_m + 2) / 3;
  for (int rr = 0; rr < nr; ++rr) {
    const int r = INV ? nr - 1 - rr : rr;
    const int sig0 = 3 * r;
    const int R = min(3, a.log_m - sig0);
    if (R == 3) ntt_round<INV, COL, 3>(a, sm, tile, sig0, tw, q);
    else if (R == 2) ntt_round<INV, COL, 2>(a, sm, tile, sig0, tw, q);
    else ntt_round<INV, COL, 1>(a, sm, tile, sig0, tw, q);
    __syncthreads();
  }

  for (uint32_t idx = threadIdx.x; idx < tilesz; idx += blockDim.x) {
    uint32_t k, x;
    if (COL) { x = idx >> a.log_k; k = idx & (a.K - 1); }
    else { k = idx >> a.log_m; x = idx & (M - 1); }
    uint64_t v = sm[pad8(idx)];
    if (a.last) {
      if (INV) v = mul_shoup_lazy(v, pr.n_inv, pr.n_inv_sh, q);
      else v = v >= q2 ? v - q2 : v;
      v = v >= q ? v - q : v;
    }
    dst[elem_index<COL>(a, tile, k, x)] = v;
  }
}

// Split of the n index bits: first (column) pass over the top n1 bits.
static int split_bits(int log_n) { return log_n <= 11 ? log_n : (log_n + 1) / 2; }

static int launch_pass(he_ctx* c, const PolyBatch& b, bool inv, bool col, int log_m, int bit_lo,
                       const uint64_t* src, uint64_t* dst, uint64_t src_stride, bool last) {
  NttPassArgs a;
  a.src = src;
  a.dst = dst;
  a.src_stride = src_stride;
  a.dst_stride = b.dst_stride;
  a.nl = b.nl;
  a.limb0 = b.limb0;
  a.level = b.level;
  a.L = (uint32_t)c->L;
  a.skip_alpha = b.skip_alpha;
  a.skip_beta = b.skip_beta ? b.skip_beta : 1;
  a.tw = reinterpret_cast<const ulonglong2*>(inv ? c->d_itw : c->d_tw);
  a.primes = c->d_primes;
  a.log_n = c->log_n;
  a.log_m = log_m;
  a.bit_lo = bit_lo;
  // transforms per CTA: 2^11 residues (256 threads, 8 residues each) and, for
  // column passes, at least 16 consecutive columns (128-byte segments)
  const int others = c->log_n - log_m;  // log2 of transforms per limb
  int log_k = 0;
  while (log_k < others && ((log_m + log_k) < 11 || (col && log_k < 4))) ++log_k;
  a.log_k = log_k;
  a.K = 1 << log_k;
  a.tiles_per_limb = 1 << (others - log_k);
  a.last = last ? 1 : 0;
  const int tilesz = 1 << (log_m + log_k);
  const int threads = tilesz >= 8 ? tilesz / 8 : 1;
  const size_t blocks = (size_t)b.npolys * b.nl * a.tiles_per_limb;
  if (blocks == 0) return HE_OK;
  if (blocks > 0x7fffffffull) return fail(HE_EINVAL, "NTT batch too large");
  const size_t smem = sizeof(uint64_t) * (tilesz + tilesz / 8);
  // algorithmic work: (N/2) * log_m butterflies and 16 N bytes per transformed limb
  double transforms = (double)b.npolys * b.nl;
  if (b.skip_alpha && c->prof_on) {
    transforms = 0;
    for (uint32_t p = 0; p < b.npolys; ++p) {
      const uint32_t j = p % a.skip_beta, lo = j * b.skip_alpha, hi = std::min(lo + b.skip_alpha, b.level);
      uint32_t skipped = 0;
      for (uint32_t t = b.limb0; t < b.limb0 + b.nl; ++t) skipped += (t >= lo && t < hi);
      transforms += b.nl - skipped;
    }
  }
  const double nn = (double)(1u << c->log_n);
  // work: the butterflies, and the inverse's scaling by N^-1 in its last pass
  const double scale = inv && last ? transforms * nn : 0.0;
  ProfScope prof(c, inv ? "intt" : "ntt", transforms * nn / 2 * log_m + scale, transforms * nn * 16, 0.0,
                 transforms * nn / 2 * log_m);
  if (inv) {
    if (col) ntt_pass_kernel<true, true><<<(unsigned)blocks, threads, smem, c->stream>>>(a);
    else ntt_pass_kernel<true, false><<<(unsigned)blocks, threads, smem, c->stream>>>(a);
  } else {
    if (col) ntt_pass_kernel<false, true><<<(unsigned)blocks, threads, smem, c->stream>>>(a);
    else ntt_pass_kernel<false, false><<<(unsigned)blocks, threads, smem, c->stream>>>(a);
  }
  HE_CUDA(cudaGetLastError());
  return HE_OK;
}

int ntt2(he_ctx* c, const PolyBatch& b, bool inv, bool* handled);

int ntt_forward(he_ctx* c, const PolyBatch& b) {
  if (!c->ntt_generic) {
    bool handled = false;
    const int rc = ntt2(c, b, false, &handled);
    if (handled) return rc;
  }
  const int n = c->log_n, n1 = split_bits(n);
  if (n1 == n) return launch_pass(c, b, false, true, n, 0, b.src, b.dst, b.src_stride, true);
  HE_TRY(launch_pass(c, b, false, true, n1, n - n1, b.src, b.dst, b.src_stride, false));
  return launch_pass(c, b, false, false, n - n1, 0, b.dst, b.dst, b.dst_stride, true);
}

int ntt_inverse(he_ctx* c, const PolyBatch& b) {
  if (!c->ntt_generic) {
    bool handled = false;
    const int rc = ntt2(c, b, true, &handled);
    if (handled) return rc;
  }
  const int n = c->log_n, n1 = split_bits(n);
  if (n1 == n) return launch_pass(c, b, true, true, n, 0, b.src, b.dst, b.src_stride, true);
  HE_TRY(launch_pass(c, b, true, false, n - n1, 0, b.src, b.dst, b.src_stride, false));
  return launch_pass(c, b, true, true, n1, n - n1, b.dst, b.dst, b.dst_stride, true);
}

}  // namespace he
