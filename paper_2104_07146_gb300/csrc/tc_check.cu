// hmle_selftest_tc_gemm: the tensor-core tile product of the mixed forms
// (tc_gemm.cuh) on a caller's matrices, so that its shared-memory layout,
// descriptors, slices and TMEM read-back can be checked on their own against
// a plain product of the same BF16 slices.
#include <cuda_runtime.h>

#include "hmle_internal.h"
#include "tc_gemm.cuh"

namespace hmle {
namespace {

// CTA c writes its copy of C = A B (column-major M x N at C + c M N).  A is
// row-major M x K, B row-major K x N.
template <int NS, bool AK, bool BK>
__global__ void __launch_bounds__(128) k_tc_check(int M, int N, int K, const double *__restrict__ A,
                                                  const double *__restrict__ B, double *__restrict__ C,
                                                  int *flags) {
  extern __shared__ double smem[];
  double *out = C + (int64_t)blockIdx.x * M * N;
  tc::gemm<NS, AK, BK>(
      M, N, K, [&](int i, int k) { return A[(int64_t)i * K + k]; },
      [&](int k, int j) { return B[(int64_t)k * N + j]; },
      [&](int i, int j, double v) { out[i + (int64_t)j * M] = v; }, smem, flags);
}

template <int NS, bool AK, bool BK>
cudaError_t launch_check(cudaStream_t st, int copies, int M, int N, int K, const double *A, const double *B,
                         double *C, int *flags) {
  const int bytes = tc::smem_words<NS>() * (int)sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_tc_check<NS, AK, BK>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  if (e != cudaSuccess) return e;
  k_tc_check<NS, AK, BK><<<copies, 128, bytes, st>>>(M, N, K, A, B, C, flags);
  return cudaGetLastError();
}

template <int NS>
cudaError_t launch_ns(cudaStream_t st, int ak, int bk, int copies, int M, int N, int K, const double *A,
                      const double *B, double *C, int *flags) {
  if (ak && bk) return launch_check<NS, true, true>(st, copies, M, N, K, A, B, C, flags);
  if (ak) return launch_check<NS, true, false>(st, copies, M, N, K, A, B, C, flags);
  if (bk) return launch_check<NS, false, true>(st, copies, M, N, K, A, B, C, flags);
  return launch_check<NS, false, false>(st, copies, M, N, K, A, B, C, flags);
}

}  // namespace
}  // namespace hmle

using namespace hmle;

struct hmle_ctx;
extern "C" __attribute__((visibility("hidden"))) cudaStream_t hmle_internal_ctx_stream(const hmle_ctx *ctx);
extern "C" __attribute__((visibility("hidden"))) hmle_status hmle_internal_ctx_fail(hmle_ctx *ctx, hmle_status s,
                                                                                   const char *msg);

extern "C" hmle_status hmle_selftest_tc_gemm(hmle_ctx *ctx, int32_t nslices, int32_t a_kfast, int32_t b_kfast,
                                             int32_t copies, int32_t M, int32_t N, int32_t K, const double *A,
                                             const double *B, double *C) {
  if (!ctx) return HMLE_ERR_INVALID_ARG;
  if (!A || !B || !C || M < 1 || N < 1 || K < 0 || copies < 1 || copies > 4096 || nslices < 1 || nslices > 3 ||
      (int64_t)M * N * copies > (1LL << 28) || (int64_t)M * K > (1LL << 28) || (int64_t)K * N > (1LL << 28))
    return hmle_internal_ctx_fail(ctx, HMLE_ERR_INVALID_ARG, "tensor-core check: bad sizes");
  cudaStream_t st = hmle_internal_ctx_stream(ctx);
  double *dA = nullptr, *dB = nullptr, *dC = nullptr;
  int *dflag = nullptr;
  int hflag = 0;
  const size_t na = (size_t)M * K, nb = (size_t)K * N, nc = (size_t)M * N * copies;
  cudaError_t e = cudaMallocAsync(&dA, sizeof(double) * (na ? na : 1), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dB, sizeof(double) * (nb ? nb : 1), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dC, sizeof(double) * nc, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dflag, sizeof(int), st);
  if (e == cudaSuccess && na) e = cudaMemcpyAsync(dA, A, sizeof(double) * na, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && nb) e = cudaMemcpyAsync(dB, B, sizeof(double) * nb, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(dflag, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    if (nslices == 1) e = launch_ns<1>(st, a_kfast, b_kfast, copies, M, N, K, dA, dB, dC, dflag);
    else if (nslices == 2) e = launch_ns<2>(st, a_kfast, b_kfast, copies, M, N, K, dA, dB, dC, dflag);
    else e = launch_ns<3>(st, a_kfast, b_kfast, copies, M, N, K, dA, dB, dC, dflag);
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(C, dC, sizeof(double) * nc, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&hflag, dflag, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(dA, st);
  cudaFreeAsync(dB, st);
  cudaFreeAsync(dC, st);
  cudaFreeAsync(dflag, st);
  if (e != cudaSuccess) return hmle_internal_ctx_fail(ctx, HMLE_ERR_CUDA, cudaGetErrorString(e));
  if (cudaStreamSynchronize(st) != cudaSuccess) return hmle_internal_ctx_fail(ctx, HMLE_ERR_CUDA, "free");
  if (hflag & kFlagTimeout)
    return hmle_internal_ctx_fail(ctx, HMLE_ERR_TIMEOUT, "a tensor-core product did not complete in time");
  return HMLE_OK;
}
