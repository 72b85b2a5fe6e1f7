// Exclusive prefix sums (int64) used to compact face, slot and row lists.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace eb {

constexpr int SCAN_BLOCK = 1024;

// per-block totals of in[0..n) (int32 or int64 values)
template <typename T>
__global__ void k_scan_block_sums(const T* __restrict__ in, int64_t n, int64_t* __restrict__ sums) {
  __shared__ int64_t s[32];
  int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int64_t v = i < n ? (int64_t)in[i] : 0;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = v;
  __syncthreads();
  if (threadIdx.x < 32) {
    int64_t w = s[threadIdx.x];
    for (int o = 16; o > 0; o >>= 1) w += __shfl_down_sync(0xffffffffu, w, o);
    if (threadIdx.x == 0) sums[blockIdx.x] = w;
  }
}

// in-place exclusive scan of a small array by one block (serial over chunks of 1024)
static __global__ void k_scan_single(int64_t* __restrict__ a, int64_t n, int64_t* __restrict__ total) {
  __shared__ int64_t s[32];
  __shared__ int64_t carry;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (int64_t base = 0; base < n; base += SCAN_BLOCK) {
    int64_t i = base + threadIdx.x;
    int64_t v = i < n ? a[i] : 0;
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int64_t x = v;
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s[w] = x;
    __syncthreads();
    if (w == 0) {
      int64_t t = s[lane];
      for (int o = 1; o < 32; o <<= 1) {
        int64_t y = __shfl_up_sync(0xffffffffu, t, o);
        if (lane >= o) t += y;
      }
      s[lane] = t;
    }
    __syncthreads();
    int64_t incl = x + (w > 0 ? s[w - 1] : 0);
    if (i < n) a[i] = carry + incl - v;
    __syncthreads();
    if (threadIdx.x == SCAN_BLOCK - 1) carry += incl;
    __syncthreads();
  }
  if (threadIdx.x == 0 && total) *total = carry;
}

// out[i] = exclusive prefix of in[i]; block offsets from k_scan_single
template <typename T>
__global__ void k_scan_apply(const T* __restrict__ in, int64_t n, const int64_t* __restrict__ boff,
                             int64_t* __restrict__ out) {
  __shared__ int64_t s[32];
  int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
  int64_t v = i < n ? (int64_t)in[i] : 0;
  int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) s[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t t = s[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(0xffffffffu, t, o);
      if (lane >= o) t += y;
    }
    s[lane] = t;
  }
  __syncthreads();
  int64_t incl = x + (w > 0 ? s[w - 1] : 0);
  if (i < n) out[i] = boff[blockIdx.x] + incl - v;
}

}  // namespace eb
