// hmle_matern_eval_noalloc: the Matern-table evaluation without any device
// allocation, for callers that cannot allocate -- a host that hands this
// library a fixed device-memory budget it must not grow, or code in a
// section where cudaMalloc is not allowed (it may synchronise the device,
// and it is refused while a stream is being captured).
//
// The scratch that the allocating entry point (hmle_matern_eval) obtains
// with cudaMallocAsync -- one Chebyshev table per value of nu -- lives here
// in a file-scope static device array instead.  Host code must not use that
// array's name as a device address: it is resolved with cudaGetSymbolAddress
// on every call made outside a stream capture (so a reset of the device's
// context, which can move the array, is followed), and a call made while the
// context's stream is being captured uses the address of the last call
// outside a capture (so the first call on a device must come before any
// capture begins).
#include <cuda_runtime.h>

#include <mutex>

#include "common.cuh"
#include "hmle_internal.h"
#include "kernels.cuh"
#include "matern.cuh"

namespace hmle {
namespace {

constexpr int kStaticNu = 16;  // at most 16 tables: 16 * 470 doubles = 60 KB per device

static __device__ __align__(256) double g_matern_scratch[kStaticNu * kTableWords];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {nullptr};

}  // namespace
}  // namespace hmle

using namespace hmle;

struct hmle_ctx;  // defined in capi.cu; its stream, device and error path are used here
extern "C" __attribute__((visibility("hidden"))) cudaStream_t hmle_internal_ctx_stream(const hmle_ctx *ctx);
extern "C" __attribute__((visibility("hidden"))) int hmle_internal_ctx_device(const hmle_ctx *ctx);
extern "C" __attribute__((visibility("hidden"))) hmle_status hmle_internal_ctx_fail(hmle_ctx *ctx, hmle_status s,
                                                                                   const char *msg);

extern "C" hmle_status hmle_matern_eval_noalloc(hmle_ctx *ctx, const double *nus, int32_t nnu,
                                                const double *x, int64_t m, double *out) {
  if (!ctx) return HMLE_ERR_INVALID_ARG;
  if (!nus || !x || !out || m < 0) return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (nnu < 1 || nnu > kStaticNu)
    return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "between 1 and 16 values of nu per call");
  for (int j = 0; j < nnu; ++j)
    if (!(nus[j] > 0.0) || !(nus[j] <= 20.0))
      return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "nu out of range");
  // the scratch address belongs to the device that owns the context's
  // stream; a call made with another device current is refused
  const int dev = hmle_internal_ctx_device(ctx);
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) return hmle_internal_ctx_fail(ctx, HMLE_ERR_CUDA, "cudaGetDevice failed");
  if (cur != dev || dev < 0 || dev >= kMaxDevices)
    return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "the context's device is not the current device");
  // inputs and outputs must already be on the device: nothing is staged
  cudaPointerAttributes ax, ao;
  if (cudaPointerGetAttributes(&ax, x) != cudaSuccess || cudaPointerGetAttributes(&ao, out) != cudaSuccess) {
    cudaGetLastError();
    return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "x and out must be device pointers");
  }
  if ((ax.type != cudaMemoryTypeDevice && ax.type != cudaMemoryTypeManaged) ||
      (ao.type != cudaMemoryTypeDevice && ao.type != cudaMemoryTypeManaged))
    return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "x and out must be device pointers");
  cudaStream_t st = hmle_internal_ctx_stream(ctx);
  bool capturing = true;   // unknown: keep the address already resolved
  {
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cap) == cudaSuccess) capturing = (cap != cudaStreamCaptureStatusNone);
    else cudaGetLastError();
  }
  double *scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev] || !capturing) {
      // with this device current; again on every call outside a capture
      double *p = nullptr;
      if (cudaGetSymbolAddress((void **)&p, g_matern_scratch) != cudaSuccess || !p) {
        cudaGetLastError();
        return hmle_internal_ctx_fail(ctx, HMLE_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed");
      }
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  cudaGetLastError();   // report only the launches below, not an earlier caller's error
  // every word of each table is written by its table kernel before the
  // evaluation kernel reads it, so nothing left by a previous call is used
  for (int j = 0; j < nnu; ++j) {
    launch_matern_table(st, nus[j], scratch + (int64_t)j * kTableWords);
    launch_matern_eval(st, scratch + (int64_t)j * kTableWords, x, m, out + (int64_t)j * m);
  }
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return hmle_internal_ctx_fail(ctx, HMLE_ERR_CUDA, cudaGetErrorString(e));
  return HMLE_OK;
}
