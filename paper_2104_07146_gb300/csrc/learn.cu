// a16: the learned start (Sec. 7 suggests precomputing the optimiser's
// initial guess).  A small perceptron maps summary statistics of one field to
// an initial theta and initial simplex steps for hmle_fit.
//
//  * Features (35): the empirical semivariogram gamma_k = mean of
//    (Z_i - Z_j)^2 / 2 over point pairs whose squared distance h^2 lies in
//    bin k, on m = min(n, 4096) points taken at caller indices
//    floor(i n / m); bins e_k <= h^2 < e_{k+1} with e_k = S 2^(k - 32),
//    S = the squared bounding-box diagonal of the sample (pairs below e_1 in
//    bin 0, h^2 = S in bin 31); log gamma_k (an empty bin takes the nearest
//    non-empty bin above it, else below), then log n, d, log sqrt(S).
//    h^2 is summed over dimensions in order with unfused multiplies and adds,
//    so every bin decision is reproducible.
//  * Perceptron 35 -> 256 (tanh) -> 256 (tanh) -> 256 (tanh) -> 8: outputs
//    are the predicted transformed coordinates of Sec. 5 (mu_1..4) and log
//    step scales (s_1..4).  Every matrix product -- the layers of the forward
//    pass, the back-propagated deltas and the weight gradients -- runs on the
//    tensor cores (tc_gemm.cuh, tcgen05.mma) with BF16 operands (the FP32
//    weights and activations rounded to BF16 as they are staged) and FP32
//    accumulation; biases, tanh, the loss and Adam are FP32.  Trained with the
//    Gaussian negative log-likelihood sum_c [exp(-2 s_c) (t_c - mu_c)^2 / 2 +
//    s_c] (batch mean) and Adam (beta1 0.9, beta2 0.999, eps 1e-8) on FP32
//    master weights.  Parameters are one flat array: W1 (256 x 35,
//    row-major), b1, W2 (256 x 256), b2, W3 (256 x 256), b3, W4 (8 x 256), b4.
//
// Every reduction runs in a fixed order: features, gradients and training
// are deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/hmle.h"
#include "common.cuh"
#include "tc_gemm.cuh"

using hmle::block_sum;

namespace {

constexpr int kBins = 32;
constexpr int kNF = 35, kNH = 256, kNO = 8, kNL = 4;
// layer l: kIn[l] -> kOut[l]; W_l at kOffW[l] (kOut x kIn, row-major), b_l after it
constexpr int kIn[kNL] = {kNF, kNH, kNH, kNH}, kOut[kNL] = {kNH, kNH, kNH, kNO};
constexpr int off_w(int l) { return l == 0 ? 0 : off_w(l - 1) + kIn[l - 1] * kOut[l - 1] + kOut[l - 1]; }
constexpr int off_b(int l) { return off_w(l) + kIn[l] * kOut[l]; }
constexpr int kNParams = off_b(kNL - 1) + kOut[kNL - 1];
static_assert(kNParams == 142856, "35-256-256-256-8");
constexpr int kTcBytes = hmle::tc::smem_words<1>() * (int)sizeof(double);
constexpr int kVarioCtas = 304;
constexpr int kVarioThreads = 128;
constexpr int kSampleMax = 4096;

// --- features ---------------------------------------------------------------
// P (SoA, d x m) and z of the sampled points
__global__ void k_vario_gather(const double *__restrict__ locs, const double *__restrict__ Z,
                               int64_t n, int d, int m, double *__restrict__ P,
                               double *__restrict__ z) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  const int64_t src = ((int64_t)i * n) / m;
  for (int k = 0; k < d; ++k) P[(int64_t)k * m + i] = locs[src * d + k];
  z[i] = Z[src];
}

// S = sum over dimensions (in order) of (max - min)^2; one CTA
__global__ void k_vario_spread(const double *__restrict__ P, int m, int d, double *__restrict__ S) {
  __shared__ double rmin[32], rmax[32];
  double acc = 0.0;
  for (int k = 0; k < d; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      lo = fmin(lo, P[(int64_t)k * m + i]);
      hi = fmax(hi, P[(int64_t)k * m + i]);
    }
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) { rmin[w] = lo; rmax[w] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {   // lo / hi hold warp 0's extremes; fold in the other warps'
      for (int q = 1; q < nw; ++q) { lo = fmin(lo, rmin[q]); hi = fmax(hi, rmax[q]); }
      const double wd = __dsub_rn(hi, lo);
      acc = __dadd_rn(acc, __dmul_rn(wd, wd));
    }
  }
  if (threadIdx.x == 0) *S = acc;
}

// Per-CTA partial histograms (sums of (dz)^2 / 2 and counts) over the pairs
// (i, j > i) of rows i = blockIdx.x, blockIdx.x + G, ...
__global__ void __launch_bounds__(kVarioThreads) k_vario_pairs(const double *__restrict__ P,
                                                               const double *__restrict__ z, int m,
                                                               int d, const double *__restrict__ Sp,
                                                               double *__restrict__ part) {
  __shared__ double red[32];
  __shared__ double edge[kBins];
  const double S = *Sp;
  if (threadIdx.x < kBins) edge[threadIdx.x] = ldexp(S, (int)threadIdx.x - 32);
  __syncthreads();
  double acc[kBins], cnt[kBins];
#pragma unroll
  for (int b = 0; b < kBins; ++b) { acc[b] = 0.0; cnt[b] = 0.0; }
  for (int i = blockIdx.x; i < m - 1; i += gridDim.x) {
    for (int j = i + 1 + threadIdx.x; j < m; j += blockDim.x) {
      double h2 = 0.0;
      for (int k = 0; k < d; ++k) {
        const double dx = __dsub_rn(P[(int64_t)k * m + i], P[(int64_t)k * m + j]);
        h2 = __dadd_rn(h2, __dmul_rn(dx, dx));
      }
      int bin = 0;
#pragma unroll
      for (int b = 1; b < kBins; ++b) bin += (edge[b] <= h2) ? 1 : 0;
      const double dz = z[i] - z[j];
      const double v = 0.5 * dz * dz;
#pragma unroll
      for (int b = 0; b < kBins; ++b) {   // register-resident histogram (no dynamic index)
        const bool hit = (b == bin);
        acc[b] += hit ? v : 0.0;
        cnt[b] += hit ? 1.0 : 0.0;
      }
    }
  }
  for (int b = 0; b < kBins; ++b) {
    const double sa = block_sum(acc[b], red);
    const double sc = block_sum(cnt[b], red);
    if (threadIdx.x == 0) {
      part[(int64_t)blockIdx.x * 2 * kBins + b] = sa;
      part[(int64_t)blockIdx.x * 2 * kBins + kBins + b] = sc;
    }
  }
}

__global__ void k_vario_final(const double *__restrict__ part, int G, double *__restrict__ out) {
  const int b = threadIdx.x;
  if (b >= 2 * kBins) return;
  double s = 0.0;
  for (int g = 0; g < G; ++g) s += part[(int64_t)g * 2 * kBins + b];
  out[b] = s;
}

// --- perceptron -------------------------------------------------------------
// X: B x 35 raw features -> Xn, standardised with mu / sd
__global__ void k_standardize(const float *__restrict__ X, const float *__restrict__ mu,
                              const float *__restrict__ sd, int B, float *__restrict__ Xn) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e < B * kNF) Xn[e] = (X[e] - mu[e % kNF]) / sd[e % kNF];
}

// out = act(in W^T + b): in B x nin, W nout x nin (row-major), out B x nout.
// CTA (x, y) computes rows 128 x .. + 127 and columns 64 y .. + 63 on the
// tensor cores (BF16 operands, FP32 accumulation).
template <bool TANH>
__global__ void __launch_bounds__(128) k_layer_fwd(const float *__restrict__ in, int nin,
                                                   const float *__restrict__ W, const float *__restrict__ b,
                                                   int nout, int B, float *__restrict__ out, int *flags) {
  extern __shared__ double smem[];
  const int m0 = blockIdx.x * hmle::tc::kTM, n0 = blockIdx.y * hmle::tc::kTN;
  hmle::tc::gemm<1, true, true>(
      min(hmle::tc::kTM, B - m0), min(hmle::tc::kTN, nout - n0), nin,
      [&](int i, int k) { return (double)in[(int64_t)(m0 + i) * nin + k]; },
      [&](int k, int j) { return (double)W[(int64_t)(n0 + j) * nin + k]; },
      [&](int i, int j, double v) {
        const float a = (float)v + b[n0 + j];
        out[(int64_t)(m0 + i) * nout + n0 + j] = TANH ? tanhf(a) : a;
      },
      smem, flags);
}

// deltas of the output layer (B x 8) and the loss of each sample; T: B x 4
__global__ void k_out_delta(const float *__restrict__ Y, const float *__restrict__ T, int B,
                            float *__restrict__ D, float *__restrict__ loss) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float l = 0.0f;
  for (int c = 0; c < 4; ++c) {
    const float mu = Y[(int64_t)b * kNO + c], s = Y[(int64_t)b * kNO + 4 + c];
    const float r = T[(int64_t)b * 4 + c] - mu, e = expf(-2.0f * s);
    D[(int64_t)b * kNO + c] = -e * r / B;
    D[(int64_t)b * kNO + 4 + c] = (1.0f - e * r * r) / B;
    l += 0.5f * e * r * r + s;
  }
  loss[b] = l;
}

// D = (Dn W) * (1 - H^2): Dn B x nn, W nn x nout (row-major), H, D B x nout
__global__ void __launch_bounds__(128) k_layer_bwd(const float *__restrict__ Dn, int nn,
                                                   const float *__restrict__ W, int nout,
                                                   const float *__restrict__ H, int B,
                                                   float *__restrict__ D, int *flags) {
  extern __shared__ double smem[];
  const int m0 = blockIdx.x * hmle::tc::kTM, n0 = blockIdx.y * hmle::tc::kTN;
  hmle::tc::gemm<1, true, false>(
      min(hmle::tc::kTM, B - m0), min(hmle::tc::kTN, nout - n0), nn,
      [&](int i, int k) { return (double)Dn[(int64_t)(m0 + i) * nn + k]; },
      [&](int k, int j) { return (double)W[(int64_t)k * nout + n0 + j]; },
      [&](int i, int j, double v) {
        const int64_t e = (int64_t)(m0 + i) * nout + n0 + j;
        const float h = H[e];
        D[e] = (float)v * (1.0f - h * h);
      },
      smem, flags);
}

// gW = D^T Hin: D B x nout, Hin B x nin, gW nout x nin (row-major); the sum
// over the batch runs on the tensor cores
__global__ void __launch_bounds__(128) k_layer_wgrad(const float *__restrict__ D, int nout,
                                                     const float *__restrict__ Hin, int nin, int B,
                                                     float *__restrict__ gW, int *flags) {
  extern __shared__ double smem[];
  const int m0 = blockIdx.x * hmle::tc::kTM, n0 = blockIdx.y * hmle::tc::kTN;
  hmle::tc::gemm<1, false, false>(
      min(hmle::tc::kTM, nout - m0), min(hmle::tc::kTN, nin - n0), B,
      [&](int i, int k) { return (double)D[(int64_t)k * nout + m0 + i]; },
      [&](int k, int j) { return (double)Hin[(int64_t)k * nin + n0 + j]; },
      [&](int i, int j, double v) { gW[(int64_t)(m0 + i) * nin + n0 + j] = (float)v; }, smem, flags);
}

// gb[j] = sum over the batch of D[b, j], in sample order
__global__ void k_bias_grad(const float *__restrict__ D, int nout, int B, float *__restrict__ gb) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nout) return;
  double s = 0.0;
  for (int b = 0; b < B; ++b) s += D[(int64_t)b * nout + j];
  gb[j] = (float)s;
}

__global__ void k_adam(float *__restrict__ p, float *__restrict__ m, float *__restrict__ v,
                       const float *__restrict__ g, int np, float lr, float bc1, float bc2) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= np) return;
  const float gq = g[q];
  const float mq = 0.9f * m[q] + 0.1f * gq;
  const float vq = 0.999f * v[q] + 0.001f * gq * gq;
  m[q] = mq;
  v[q] = vq;
  p[q] -= lr * (mq / bc1) / (sqrtf(vq / bc2) + 1e-8f);
}

// rows idx[0..B) of src (ld columns) -> dst
__global__ void k_gather_rows(const float *__restrict__ src, const int32_t *__restrict__ idx,
                              int B, int ld, float *__restrict__ dst) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= B * ld) return;
  const int b = e / ld, c = e % ld;
  dst[e] = src[(int64_t)idx[b] * ld + c];
}

__global__ void k_sum_f(const float *__restrict__ x, int n, float *__restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) s += x[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = (float)s;
}

uint64_t splitmix(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

}  // namespace

struct hmle_mlp {
  float *p = nullptr, *m = nullptr, *v = nullptr;   // parameters, Adam moments (device)
  float mu[kNF], sd[kNF];                           // feature standardisation
  int64_t t = 0;                                    // Adam step count
};

namespace {

struct Scratch {   // per-call device buffers for B samples
  float *X = nullptr, *Xn, *H[kNL], *T, *D[kNL], *loss, *g, *mu, *sd, *lsum;
  int32_t *idx = nullptr;
  int *flags = nullptr;   // error word of the tensor-core products (kFlagTimeout)
};

cudaError_t scratch_alloc(Scratch &s, int B, cudaStream_t st) {
  size_t acts = 0;
  for (int l = 0; l < kNL; ++l) acts += 2 * (size_t)kOut[l];
  const size_t fl = (size_t)B * (2 * kNF + acts + 4 + 1) + kNParams + 2 * kNF + 1;
  float *base = nullptr;
  cudaError_t e = cudaMallocAsync(&base, fl * sizeof(float), st);
  if (e != cudaSuccess) return e;
  e = cudaMallocAsync(&s.idx, sizeof(int32_t) * std::max(B, 1) + 16, st);
  if (e != cudaSuccess) { cudaFreeAsync(base, st); return e; }
  s.flags = reinterpret_cast<int *>(s.idx + std::max(B, 1));
  e = cudaMemsetAsync(s.flags, 0, sizeof(int), st);
  float *q = base;
  s.X = q; q += (size_t)B * kNF;
  s.Xn = q; q += (size_t)B * kNF;
  for (int l = 0; l < kNL; ++l) { s.H[l] = q; q += (size_t)B * kOut[l]; }
  for (int l = 0; l < kNL; ++l) { s.D[l] = q; q += (size_t)B * kOut[l]; }
  s.T = q; q += (size_t)B * 4;
  s.loss = q; q += B;
  s.g = q; q += kNParams;
  s.mu = q; q += kNF;
  s.sd = q; q += kNF;
  s.lsum = q;
  return e;
}

void scratch_free(Scratch &s, cudaStream_t st) {
  if (s.X) cudaFreeAsync(s.X, st);
  if (s.idx) cudaFreeAsync(s.idx, st);
  s = Scratch{};
}

dim3 tiles(int rows, int cols) {
  return dim3((rows + hmle::tc::kTM - 1) / hmle::tc::kTM, (cols + hmle::tc::kTN - 1) / hmle::tc::kTN);
}

void launch_fwd(cudaStream_t st, const hmle_mlp *M, const Scratch &s, int B);

void launch_grad(cudaStream_t st, const hmle_mlp *M, const Scratch &s, int B);

hmle_status cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return HMLE_OK;
  cudaGetLastError();
  return e == cudaErrorMemoryAllocation ? HMLE_ERR_OOM : HMLE_ERR_CUDA;
}

// the products' error word after a synchronisation: TIMEOUT if a bounded wait
// of the tensor cores ran out
hmle_status flag_status(const Scratch &s, cudaStream_t st) {
  int f = 0;
  cudaError_t e = cudaMemcpyAsync(&f, s.flags, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  return (f & hmle::kFlagTimeout) ? HMLE_ERR_TIMEOUT : HMLE_OK;
}

cudaStream_t ctx_stream(hmle_ctx *ctx);

}  // namespace

extern "C" __attribute__((visibility("hidden"))) cudaStream_t hmle_internal_ctx_stream(const hmle_ctx *ctx);

namespace {
cudaStream_t ctx_stream(hmle_ctx *ctx) { return hmle_internal_ctx_stream(ctx); }

bool is_dev(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}
}  // namespace

namespace {

void launch_fwd(cudaStream_t st, const hmle_mlp *M, const Scratch &s, int B) {
  k_standardize<<<(B * kNF + 255) / 256, 256, 0, st>>>(s.X, s.mu, s.sd, B, s.Xn);
  const float *in = s.Xn;
  for (int l = 0; l < kNL; ++l) {
    const bool last = l == kNL - 1;
    const float *W = M->p + off_w(l), *b = M->p + off_b(l);
    if (last)
      k_layer_fwd<false><<<tiles(B, kOut[l]), 128, kTcBytes, st>>>(in, kIn[l], W, b, kOut[l], B, s.H[l], s.flags);
    else
      k_layer_fwd<true><<<tiles(B, kOut[l]), 128, kTcBytes, st>>>(in, kIn[l], W, b, kOut[l], B, s.H[l], s.flags);
    in = s.H[l];
  }
}

// forward, output deltas, then per layer (last to first): weight gradient,
// bias gradient, and the deltas of the layer below
void launch_grad(cudaStream_t st, const hmle_mlp *M, const Scratch &s, int B) {
  launch_fwd(st, M, s, B);
  k_out_delta<<<(B + 127) / 128, 128, 0, st>>>(s.H[kNL - 1], s.T, B, s.D[kNL - 1], s.loss);
  for (int l = kNL - 1; l >= 0; --l) {
    const float *Hin = l == 0 ? s.Xn : s.H[l - 1];
    k_layer_wgrad<<<tiles(kOut[l], kIn[l]), 128, kTcBytes, st>>>(s.D[l], kOut[l], Hin, kIn[l], B,
                                                                 s.g + off_w(l), s.flags);
    k_bias_grad<<<(kOut[l] + 127) / 128, 128, 0, st>>>(s.D[l], kOut[l], B, s.g + off_b(l));
    if (l > 0)
      k_layer_bwd<<<tiles(B, kIn[l]), 128, kTcBytes, st>>>(s.D[l], kOut[l], M->p + off_w(l), kIn[l],
                                                           s.H[l - 1], B, s.D[l - 1], s.flags);
  }
  k_sum_f<<<1, 256, 0, st>>>(s.loss, B, s.lsum);
}

// dynamic shared memory of the tensor-core kernels (above 48 KB): once
cudaError_t mlp_setup() {
  static std::once_flag once;
  static cudaError_t err = cudaSuccess;
  std::call_once(once, [] {
    err = cudaFuncSetAttribute(k_layer_fwd<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcBytes);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_layer_fwd<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcBytes);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_layer_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcBytes);
    if (err == cudaSuccess)
      err = cudaFuncSetAttribute(k_layer_wgrad, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcBytes);
  });
  return err;
}

}  // namespace

extern "C" {

int32_t hmle_mlp_nparams(void) { return kNParams; }

hmle_status hmle_mlp_create(hmle_ctx *ctx, uint64_t seed, hmle_mlp **out) {
  if (!ctx || !out) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  hmle_mlp *M = new (std::nothrow) hmle_mlp();
  if (!M) return HMLE_ERR_OOM;
  // weights uniform in +-1/sqrt(fan_in) from a counter-based generator,
  // biases 0; no standardisation until hmle_mlp_train / hmle_mlp_set
  std::vector<float> p(kNParams, 0.0f);
  auto fill = [&](int off, int rows, int cols) {
    const double a = 1.0 / std::sqrt((double)cols);
    for (int i = 0; i < rows * cols; ++i) {
      const double u = (double)(splitmix(seed ^ splitmix((uint64_t)(off + i))) >> 11) * 0x1.0p-53;
      p[off + i] = (float)((2.0 * u - 1.0) * a);
    }
  };
  for (int l = 0; l < kNL; ++l) fill(off_w(l), kOut[l], kIn[l]);
  for (int k = 0; k < kNF; ++k) { M->mu[k] = 0.0f; M->sd[k] = 1.0f; }
  cudaError_t e = cudaMallocAsync(&M->p, 3 * sizeof(float) * kNParams, st);
  if (e == cudaSuccess) {
    M->m = M->p + kNParams;
    M->v = M->m + kNParams;
    e = cudaMemcpyAsync(M->p, p.data(), sizeof(float) * kNParams, cudaMemcpyHostToDevice, st);
  }
  if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, 2 * sizeof(float) * kNParams, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    if (M->p) cudaFree(M->p);
    delete M;
    return cuda_status(e);
  }
  *out = M;
  return HMLE_OK;
}

void hmle_mlp_destroy(hmle_mlp *M) {
  if (!M) return;
  if (M->p) cudaFree(M->p);
  delete M;
}

hmle_status hmle_mlp_set(hmle_ctx *ctx, hmle_mlp *M, const float *params, const float *mu,
                         const float *sd) {
  if (!ctx || !M) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  if (mu) std::memcpy(M->mu, mu, sizeof(M->mu));
  if (sd) {
    for (int k = 0; k < kNF; ++k)
      if (!(sd[k] > 0.0f)) return HMLE_ERR_INVALID_ARG;
    std::memcpy(M->sd, sd, sizeof(M->sd));
  }
  if (params) {
    cudaError_t e = cudaMemcpyAsync(M->p, params, sizeof(float) * kNParams, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(M->m, 0, 2 * sizeof(float) * kNParams, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
    M->t = 0;
  }
  return HMLE_OK;
}

hmle_status hmle_mlp_get(hmle_ctx *ctx, const hmle_mlp *M, float *params, float *mu, float *sd) {
  if (!ctx || !M) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  if (mu) std::memcpy(mu, M->mu, sizeof(M->mu));
  if (sd) std::memcpy(sd, M->sd, sizeof(M->sd));
  if (params) {
    cudaError_t e = cudaMemcpyAsync(params, M->p, sizeof(float) * kNParams, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return HMLE_OK;
}

hmle_status hmle_mlp_forward(hmle_ctx *ctx, const hmle_mlp *M, const float *feats, int32_t m,
                             float *out) {
  if (!ctx || !M || !feats || !out || m < 1) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  Scratch s;
  cudaError_t e = mlp_setup();
  if (e == cudaSuccess) e = scratch_alloc(s, m, st);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(s.X, feats, sizeof(float) * m * kNF, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.mu, M->mu, sizeof(M->mu), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.sd, M->sd, sizeof(M->sd), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    launch_fwd(st, M, s, m);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaMemcpyAsync(out, s.H[kNL - 1], sizeof(float) * m * kNO, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  const hmle_status fs = e == cudaSuccess ? flag_status(s, st) : cuda_status(e);
  scratch_free(s, st);
  cudaStreamSynchronize(st);
  return fs;
}

hmle_status hmle_mlp_grad(hmle_ctx *ctx, const hmle_mlp *M, const float *feats,
                          const float *targets, int32_t m, float *grad, float *loss) {
  if (!ctx || !M || !feats || !targets || m < 1) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  Scratch s;
  cudaError_t e = mlp_setup();
  if (e == cudaSuccess) e = scratch_alloc(s, m, st);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(s.X, feats, sizeof(float) * m * kNF, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.T, targets, sizeof(float) * m * 4, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.mu, M->mu, sizeof(M->mu), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.sd, M->sd, sizeof(M->sd), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    launch_grad(st, M, s, m);
    e = cudaGetLastError();
  }
  float l = 0.0f;
  if (e == cudaSuccess && grad) e = cudaMemcpyAsync(grad, s.g, sizeof(float) * kNParams, cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&l, s.lsum, sizeof(float), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (loss) *loss = l / m;
  const hmle_status fs = e == cudaSuccess ? flag_status(s, st) : cuda_status(e);
  scratch_free(s, st);
  cudaStreamSynchronize(st);
  return fs;
}

hmle_status hmle_mlp_adam_step(hmle_ctx *ctx, hmle_mlp *M, const float *grad, float lr) {
  if (!ctx || !M || !grad) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  float *g = nullptr;
  cudaError_t e = cudaMallocAsync(&g, sizeof(float) * kNParams, st);
  if (e != cudaSuccess) return cuda_status(e);
  e = cudaMemcpyAsync(g, grad, sizeof(float) * kNParams, cudaMemcpyDefault, st);
  M->t += 1;
  const float bc1 = (float)(1.0 - std::pow(0.9, (double)M->t));
  const float bc2 = (float)(1.0 - std::pow(0.999, (double)M->t));
  if (e == cudaSuccess) {
    k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(M->p, M->m, M->v, g, kNParams, lr, bc1, bc2);
    e = cudaGetLastError();
  }
  cudaFreeAsync(g, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  return cuda_status(e);
}

hmle_status hmle_mlp_train(hmle_ctx *ctx, hmle_mlp *M, const float *feats, const float *targets,
                           int32_t m, int32_t epochs, int32_t batch, float lr, uint64_t seed,
                           float *loss_first, float *loss_last) {
  if (!ctx || !M || !feats || !targets || m < 1 || epochs < 1 || batch < 1 || !(lr > 0.0f))
    return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  batch = std::min(batch, m);
  {
    const cudaError_t e0 = mlp_setup();
    if (e0 != cudaSuccess) return cuda_status(e0);
  }
  // standardisation from the training features (host, double)
  std::vector<float> F((size_t)m * kNF), Tg((size_t)m * 4);
  cudaError_t e = cudaMemcpyAsync(F.data(), feats, sizeof(float) * F.size(), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Tg.data(), targets, sizeof(float) * Tg.size(), cudaMemcpyDefault, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  for (int k = 0; k < kNF; ++k) {
    double s = 0.0, s2 = 0.0;
    for (int i = 0; i < m; ++i) s += F[(size_t)i * kNF + k];
    const double mean = s / m;
    for (int i = 0; i < m; ++i) {
      const double dv = F[(size_t)i * kNF + k] - mean;
      s2 += dv * dv;
    }
    M->mu[k] = (float)mean;
    M->sd[k] = (float)std::max(std::sqrt(s2 / m), 1e-3);
  }
  // the whole training set and the batch buffers on the device
  float *Fd = nullptr, *Td = nullptr;
  Scratch s;
  e = cudaMallocAsync(&Fd, sizeof(float) * F.size(), st);
  if (e == cudaSuccess) e = cudaMallocAsync(&Td, sizeof(float) * Tg.size(), st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Fd, F.data(), sizeof(float) * F.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(Td, Tg.data(), sizeof(float) * Tg.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = scratch_alloc(s, batch, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.mu, M->mu, sizeof(M->mu), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(s.sd, M->sd, sizeof(M->sd), cudaMemcpyHostToDevice, st);
  std::vector<int32_t> perm(m), idx(batch);
  for (int i = 0; i < m; ++i) perm[i] = i;
  float lf = 0.0f, ll = 0.0f;
  for (int ep = 0; ep < epochs && e == cudaSuccess; ++ep) {
    // deterministic shuffle (Fisher-Yates with a counter-based generator)
    for (int i = m - 1; i > 0; --i) {
      const uint64_t r = splitmix(seed ^ splitmix(((uint64_t)ep << 32) | (uint64_t)i));
      std::swap(perm[i], perm[(int)(r % (uint64_t)(i + 1))]);
    }
    double esum = 0.0;
    int nb = 0;
    for (int b0 = 0; b0 + batch <= m && e == cudaSuccess; b0 += batch) {
      for (int k = 0; k < batch; ++k) idx[k] = perm[b0 + k];
      e = cudaMemcpyAsync(s.idx, idx.data(), sizeof(int32_t) * batch, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) break;
      k_gather_rows<<<(batch * kNF + 255) / 256, 256, 0, st>>>(Fd, s.idx, batch, kNF, s.X);
      k_gather_rows<<<(batch * 4 + 255) / 256, 256, 0, st>>>(Td, s.idx, batch, 4, s.T);
      launch_grad(st, M, s, batch);
      M->t += 1;
      const float bc1 = (float)(1.0 - std::pow(0.9, (double)M->t));
      const float bc2 = (float)(1.0 - std::pow(0.999, (double)M->t));
      k_adam<<<(kNParams + 255) / 256, 256, 0, st>>>(M->p, M->m, M->v, s.g, kNParams, lr, bc1, bc2);
      float l = 0.0f;
      e = cudaMemcpyAsync(&l, s.lsum, sizeof(float), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      esum += l / batch;
      ++nb;
    }
    const float el = nb ? (float)(esum / nb) : 0.0f;
    if (ep == 0) lf = el;
    ll = el;
  }
  if (loss_first) *loss_first = lf;
  if (loss_last) *loss_last = ll;
  const hmle_status fs = (e == cudaSuccess && s.flags) ? flag_status(s, st) : cuda_status(e);
  scratch_free(s, st);
  if (Fd) cudaFreeAsync(Fd, st);
  if (Td) cudaFreeAsync(Td, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  return fs != HMLE_OK ? fs : cuda_status(e2);
}

hmle_status hmle_features(hmle_ctx *ctx, const double *locs, int64_t n, int32_t d, const double *Z,
                          float *feat) {
  if (!ctx || !locs || !Z || !feat || n < 2 || (d != 2 && d != 3)) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = ctx_stream(ctx);
  const int m = (int)std::min<int64_t>(n, kSampleMax);
  double *L = nullptr, *Zd = nullptr, *P = nullptr, *z = nullptr, *part = nullptr, *out = nullptr;
  const bool ldev = is_dev(locs), zdev = is_dev(Z);
  const size_t words = (ldev ? 0 : (size_t)n * d) + (zdev ? 0 : (size_t)n) + (size_t)m * (d + 1) +
                       (size_t)kVarioCtas * 2 * kBins + 2 * kBins + 1;
  double *pool = nullptr;
  cudaError_t e = cudaMallocAsync(&pool, sizeof(double) * words, st);
  if (e != cudaSuccess) return cuda_status(e);
  double *q = pool;
  if (!ldev) { L = q; q += (size_t)n * d; } else { L = const_cast<double *>(locs); }
  if (!zdev) { Zd = q; q += (size_t)n; } else { Zd = const_cast<double *>(Z); }
  P = q; q += (size_t)m * d;
  z = q; q += m;
  part = q; q += (size_t)kVarioCtas * 2 * kBins;
  out = q; q += 2 * kBins;
  double *S = q;
  if (!ldev) e = cudaMemcpyAsync(L, locs, sizeof(double) * n * d, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess && !zdev) e = cudaMemcpyAsync(Zd, Z, sizeof(double) * n, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) {
    k_vario_gather<<<(m + 255) / 256, 256, 0, st>>>(L, Zd, n, d, m, P, z);
    k_vario_spread<<<1, 256, 0, st>>>(P, m, d, S);
    k_vario_pairs<<<kVarioCtas, kVarioThreads, 0, st>>>(P, z, m, d, S, part);
    k_vario_final<<<1, 64, 0, st>>>(part, kVarioCtas, out);
    e = cudaGetLastError();
  }
  double h[2 * kBins + 1];
  if (e == cudaSuccess) e = cudaMemcpyAsync(h, out, sizeof(double) * (2 * kBins + 1), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(pool, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_status(e);
  const double *sum = h, *cnt = h + kBins;
  const double Sv = h[2 * kBins];
  for (int k = 0; k < kBins; ++k) {
    int src = k;
    if (!(cnt[src] > 0.0)) {
      src = -1;
      for (int j = k + 1; j < kBins && src < 0; ++j) if (cnt[j] > 0.0) src = j;
      for (int j = k - 1; j >= 0 && src < 0; --j) if (cnt[j] > 0.0) src = j;
    }
    const double g = src >= 0 ? sum[src] / cnt[src] : 0.0;
    feat[k] = (float)(g > 0.0 ? std::log(g) : 0.0);
  }
  feat[32] = (float)std::log((double)n);
  feat[33] = (float)d;
  feat[34] = (float)(Sv > 0.0 ? 0.5 * std::log(Sv) : 0.0);
  return HMLE_OK;
}

}  // extern "C"
