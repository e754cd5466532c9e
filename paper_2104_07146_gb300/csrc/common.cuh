// Device helpers shared by the libhmle kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace hmle {

// Error flags raised by kernels (bit mask in one device int).
constexpr int kFlagNotSpd = 1;
constexpr int kFlagRankOverflow = 2;
constexpr int kFlagNonFinite = 4;
constexpr int kFlagTimeout = 8;    // a bounded wait on the tensor cores ran out

__device__ __forceinline__ void raise_flag(int *flags, int f) { atomicOr(flags, f); }

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum for blockDim.x <= 1024; red must hold 32 doubles.  Result
// returned to every thread.  Fixed reduction order (deterministic).
__device__ __forceinline__ double block_sum(double v, double *red) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[wid] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < nw; ++w) s += red[w];
  __syncthreads();
  return s;
}

// Block-wide argmax of |v| (ties -> lowest index).  Returns the index and the
// signed value at that index.
__device__ __forceinline__ void block_argmax_abs(double v, int idx, double *redv,
                                                 int *redi, double *out_v, int *out_i) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = (blockDim.x + 31) >> 5;
  double a = fabs(v);
  for (int o = 16; o > 0; o >>= 1) {
    double a2 = __shfl_xor_sync(0xffffffffu, a, o);
    double v2 = __shfl_xor_sync(0xffffffffu, v, o);
    int i2 = __shfl_xor_sync(0xffffffffu, idx, o);
    if (a2 > a || (a2 == a && i2 < idx)) { a = a2; v = v2; idx = i2; }
  }
  __syncthreads();
  if (lane == 0) { redv[wid] = v; redi[wid] = idx; }
  __syncthreads();
  double bv = redv[0];
  int bi = redi[0];
  for (int w = 1; w < nw; ++w) {
    double aw = fabs(redv[w]);
    if (aw > fabs(bv) || (aw == fabs(bv) && redi[w] < bi)) { bv = redv[w]; bi = redi[w]; }
  }
  __syncthreads();
  *out_v = bv;
  *out_i = bi;
}

// SplitMix64 output function (Steele, Lea, Flood 2014) as a hash.
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

// Counter-based random sign for entry (i, j) of the sampling matrix of
// block `blk`: +1 or -1.
__device__ __forceinline__ double rademacher(uint64_t seed, int64_t blk, int64_t i, int64_t j) {
  uint64_t z = seed + (uint64_t)blk * 0x9E3779B97F4A7C15ull +
               (uint64_t)i * 0xD1B54A32D192ED03ull + (uint64_t)j * 0x8CB92BA72F3D8DD7ull;
  return (mix64(z) >> 63) ? -1.0 : 1.0;
}

}  // namespace hmle
