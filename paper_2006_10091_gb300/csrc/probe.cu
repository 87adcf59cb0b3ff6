// probe.cu -- register-resident integer throughput probes behind the integer
// roof the benchmark reports: chains of 32-bit multiply-adds, chains of 64-bit
// Shoup products (w known: a*w - umulhi(a, w')*q), radix-8 rounds of the
// lazy forward butterfly, 64 x 64 -> 128-bit multiply-accumulates, and the
// split (Karatsuba) key products of residues below 2^40.  No memory traffic inside the timed loops; every
// thread writes one word at the end (the output buffer holds exactly one word
// per thread).
#include <cuda_runtime.h>
#include <stdint.h>

#include "he_common.cuh"
#include "he_internal.h"

namespace he {

__global__ void probe_imad(uint32_t* out, int iters) {
  uint32_t a[8];
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x + k;
  const uint32_t m = 0x9E3779B9u, c = blockIdx.x;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 16; ++u)
#pragma unroll
      for (int k = 0; k < 8; ++k) a[k] = a[k] * m + c;
  }
  uint32_t r = 0;
  for (int k = 0; k < 8; ++k) r ^= a[k];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

__global__ void probe_shoup(uint64_t* out, int iters, uint64_t q, uint64_t w, uint64_t wsh) {
  uint64_t x[4];
  for (int k = 0; k < 4; ++k) x[k] = threadIdx.x + 6u * k + 1;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int k = 0; k < 4; ++k) x[k] = mul_shoup_lazy(x[k], w, wsh, q);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = x[0] ^ x[1] ^ x[2] ^ x[3];
}

__global__ void probe_bfly(uint64_t* out, int iters, uint64_t q, const uint64_t* tw) {
  uint64_t v[8], w[7], ws[7];
  for (int j = 0; j < 8; ++j) v[j] = (threadIdx.x * 8u + j + blockIdx.x) % q;
  for (int j = 0; j < 7; ++j) {
    w[j] = tw[2 * j];
    ws[j] = tw[2 * j + 1];
  }
  const uint64_t q2 = q + q;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int st = 0; st < 3; ++st) {
      const int half = 8 >> (st + 1);
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        if (j & half) continue;
        const int ti = (1 << st) - 1 + (j >> (3 - st));
        uint64_t X = v[j];
        X = X >= q2 ? X - q2 : X;  // keeps the values bounded over the loop
        const uint64_t t = mul_shoup_lazy(v[j + half], w[ti], ws[ti], q);
        v[j] = X + t;
        v[j + half] = X + q2 + q2 - t;
      }
    }
  }
  uint64_t r = 0;
  for (int j = 0; j < 8; ++j) r ^= v[j];
  out[blockIdx.x * blockDim.x + threadIdx.x] = r;
}

// 64 x 64 -> 128-bit multiply-accumulates (the key products of the fused
// key switch, summed unreduced): four independent 128-bit sums per thread,
// 32 products per iteration; the eight first operands are perturbed by the
// sums after every iteration, so that no product is the same from one
// iteration to the next (a loop-invariant product could be computed once).
__global__ void probe_mac(uint64_t* out, int iters, uint64_t q) {
  uint64_t x[8], y[4], lo[4] = {0, 0, 0, 0}, hi[4] = {0, 0, 0, 0};
  for (int k = 0; k < 8; ++k) x[k] = (0x9E3779B97F4A7C15ull * (threadIdx.x + 8u * k + 1)) % q;
  for (int k = 0; k < 4; ++k) y[k] = (0xC2B2AE3D27D4EB4Full * (blockIdx.x + 8u * k + 3)) % q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u)
#pragma unroll
      for (int k = 0; k < 4; ++k) mac128(lo[k], hi[k], x[u], y[k]);
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] += lo[u & 3] & 0xFF;
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (lo[0] ^ lo[1] ^ lo[2] ^ lo[3]) + (hi[0] ^ hi[1] ^ hi[2] ^ hi[3]) % q;
}

// The split key products of the fused key switch on primes below 2^40
// (mac_split3: three 32 x 32 -> 64-bit multiply-adds into 64-bit sums per
// product, no carries), laid out like probe_mac: four second operands split
// once, eight first operands perturbed and split again after every iteration.
__global__ void probe_mac3(uint64_t* out, int iters, uint64_t q) {
  constexpr uint32_t sb = 20, mask = (1u << sb) - 1;
  uint64_t x[8], ll[4] = {0, 0, 0, 0}, hh[4] = {0, 0, 0, 0}, ss[4] = {0, 0, 0, 0};
  Split3 ys[4];
  for (int k = 0; k < 8; ++k) x[k] = (0x9E3779B97F4A7C15ull * (threadIdx.x + 8u * k + 1)) % q;
  for (int k = 0; k < 4; ++k) ys[k] = split3((0xC2B2AE3D27D4EB4Full * (blockIdx.x + 8u * k + 3)) % q, sb, mask);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const Split3 xs = split3(x[u], sb, mask);
#pragma unroll
      for (int k = 0; k < 4; ++k) mac_split3(ll[k], hh[k], ss[k], xs, ys[k]);
    }
#pragma unroll
    for (int u = 0; u < 8; ++u) x[u] = (x[u] + (ll[u & 3] & 0xFF)) & ((1ull << 40) - 1);
  }
  out[blockIdx.x * blockDim.x + threadIdx.x] = (ll[0] ^ hh[1] ^ ss[2] ^ ll[3]) + (hh[0] ^ ss[1] ^ ll[2] ^ ss[3]) % q;
}

}  // namespace he

using namespace he;

extern "C" int he_probe_alu(int kind, double* per_clock_per_sm, double* per_second) {
  if (kind < 0 || kind > 4 || !per_clock_per_sm || !per_second) return fail(HE_EINVAL, "he_probe_alu: bad argument");
  int dev = 0, sms = 0, khz = 0;
  HE_CUDA(cudaGetDevice(&dev));
  HE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  HE_CUDA(cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, dev));
  const int blocks = sms * 8, threads = 256;
  void* out = nullptr;
  uint64_t* tw = nullptr;
  HE_CUDA(cudaMalloc(&out, sizeof(uint64_t) * blocks * threads));
  const uint64_t q = (1ull << 40) - 87;  // odd, < 2^40
  uint64_t htw[14];
  for (int j = 0; j < 7; ++j) {
    htw[2 * j] = (0x9E3779B97F4A7C15ull * (uint64_t)(j + 1)) % q;
    htw[2 * j + 1] = (uint64_t)(((unsigned __int128)htw[2 * j] << 64) / q);
  }
  if (cudaMalloc(&tw, sizeof(htw)) != cudaSuccess || cudaMemcpy(tw, htw, sizeof(htw), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(out);
    cudaFree(tw);
    return fail(HE_ECUDA, "he_probe_alu: allocation");
  }
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  float ms = 0.f;
  double ops = 0;
  for (int rep = 0; rep < 2; ++rep) {  // the second run is timed
    cudaEventRecord(e0);
    if (kind == 0) {
      probe_imad<<<blocks, threads>>>((uint32_t*)out, 4096);
      ops = (double)blocks * threads * 4096 * 16 * 8;
    } else if (kind == 1) {
      probe_shoup<<<blocks, threads>>>((uint64_t*)out, 1024, q, htw[0], htw[1]);
      ops = (double)blocks * threads * 1024 * 8 * 4;
    } else if (kind == 2) {
      probe_bfly<<<blocks, threads>>>((uint64_t*)out, 2000, q, tw);
      ops = (double)blocks * threads * 2000 * 12;
    } else if (kind == 3) {
      probe_mac<<<blocks, threads>>>((uint64_t*)out, 1024, q);
      ops = (double)blocks * threads * 1024 * 8 * 4;
    } else {
      probe_mac3<<<blocks, threads>>>((uint64_t*)out, 1024, q);
      ops = (double)blocks * threads * 1024 * 8 * 4;
    }
    cudaEventRecord(e1);
  }
  const cudaError_t err = cudaEventSynchronize(e1);
  if (err == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(out);
  cudaFree(tw);
  if (err != cudaSuccess || ms <= 0.f) return fail(HE_ECUDA, "he_probe_alu: timing");
  *per_second = ops / (ms * 1e-3);
  *per_clock_per_sm = *per_second / ((double)sms * khz * 1e3);
  return HE_OK;
}
