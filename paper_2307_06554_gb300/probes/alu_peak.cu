// Integer-pipe throughput microbenchmark: the ALU ceilings against which the
// NTT path's roofline is reported.  Each thread runs 8 independent chains of
// one operation (no memory traffic inside the loop); the grid fills every SM.
#include <cstdint>
#include <cstdio>
#include <cuda_runtime.h>

#define CHAINS 8
#define UNROLL 16

template <int OP>
__global__ void k_probe(uint64_t* out, uint64_t w, uint64_t wp, uint64_t q, int iters) {
  uint32_t x[CHAINS];
  uint64_t y[CHAINS];
  for (int j = 0; j < CHAINS; ++j) {
    x[j] = threadIdx.x * 131u + j;
    y[j] = threadIdx.x * 131ull + j;
  }
  const uint32_t w32 = (uint32_t)w, wp32 = (uint32_t)wp, q32 = (uint32_t)q;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int u = 0; u < UNROLL; ++u)
#pragma unroll
      for (int j = 0; j < CHAINS; ++j) {
        if (OP == 0) x[j] = x[j] * w32 + wp32;                                       // IMAD
        if (OP == 1) x[j] = __umulhi(x[j], wp32) ^ x[j];                             // IMAD.HI (+LOP)
        if (OP == 2) x[j] = x[j] * w32 - __umulhi(x[j], wp32) * q32;                 // 32-bit Shoup
        if (OP == 3) y[j] = y[j] * w - __umul64hi(y[j], wp) * q;                     // 64-bit Shoup
        if (OP == 4) x[j] = x[j] * w32 - ((x[j] * wp32) >> 16) * q32;                // Shoup, 16-bit quotient
      }
  }
  uint64_t r = 0;
  for (int j = 0; j < CHAINS; ++j) r ^= x[j] ^ y[j];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = r;
}

int main() {
  int sms = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int threads = 256, blocks = sms * 8, iters = 2048;
  uint64_t* out = nullptr;
  if (cudaMalloc(&out, sizeof(uint64_t) * threads * blocks) != cudaSuccess) return 1;
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  const double ops = (double)threads * blocks * iters * UNROLL * CHAINS;
  const char* names[] = {"imad32", "imad32_hi", "shoup32_mulmod", "shoup64_mulmod", "shoup16q_mulmod"};
  // 12289 with w = 5000; 59-bit prime 288230376151760897 with w = 2^40 + 7
  const uint64_t W32 = 5000, WP32 = (uint64_t)((5000ull << 32) / 12289), Q32 = 12289;
  const uint64_t Q64 = 288230376151760897ull, W64 = (1ull << 40) + 7;
  const uint64_t WP64 = (uint64_t)(((unsigned __int128)W64 << 64) / Q64);
  printf("{\"sms\": %d, \"results\": [", sms);
  const uint64_t WP16 = (5000ull << 16) / 12289;  // x stays below 2q < 2^16 along each chain
  for (int op = 0; op < 5; ++op) {
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      cudaEventRecord(e0);
      if (op == 0) k_probe<0><<<blocks, threads>>>(out, W32, WP32, Q32, iters);
      if (op == 1) k_probe<1><<<blocks, threads>>>(out, W32, WP32, Q32, iters);
      if (op == 2) k_probe<2><<<blocks, threads>>>(out, W32, WP32, Q32, iters);
      if (op == 3) k_probe<3><<<blocks, threads>>>(out, W64, WP64, Q64, iters / 4);
      if (op == 4) k_probe<4><<<blocks, threads>>>(out, W32, WP16, Q32, iters);
      cudaEventRecord(e1);
      cudaEventSynchronize(e1);
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms < best) best = ms;
    }
    const double n = op == 3 ? ops / 4 : ops;
    printf("%s{\"op\": \"%s\", \"per_s\": %.4e}", op ? ", " : "", names[op], n / (best * 1e-3));
  }
  printf("], \"error\": \"%s\"}\n", cudaGetErrorString(cudaGetLastError()));
  cudaFree(out);
  return 0;
}
