// a10-a11 as one persistent kernel each: the forward sweep w <- L~^{-1} w and
// the backward sweep v <- L~^{-T} v on one vector (cluster order), for the
// preconditioner of the PCG and for hmle_solve.
//
// The sweep launched kernel by kernel costs three small launches per leaf
// (thousands per solve), and each launch carries a few microseconds of GPU
// latency whatever its work.  Here one cooperative launch runs every leaf:
// per leaf (in sweep order)
//   A  the diagonal leaf's triangular solve (one warp of CTA 0),
//   B  the coupling vectors of the leaf's low-rank blocks, one task per CTA
//      (forward: h_A = W_A^T w[cols A] for the blocks whose columns end at
//      the leaf; backward: h_A = U_A^T v[rows A] for those whose rows start
//      there),
//   C  the updates of the affected leaf rows (forward) or column leaves
//      (backward), one leaf per CTA, each a fixed-order sum,
// separated by grid barriers.  The vector and the coupling vectors change
// during the launch, so they are read through L2 (ld.global.cg), never from
// an SM's L1.  The barrier waits are bounded: a wait that
// runs out sets an error word, every CTA then leaves at its next barrier,
// and the host reports HMLE_ERR_TIMEOUT.
#include <cuda_runtime.h>

#include <algorithm>
#include <mutex>

#include "common.cuh"
#include "hmle_internal.h"
#include "kernels.cuh"

namespace hmle {
namespace {

constexpr int kSolveThreads = 128;
constexpr long long kBarrierSpins = 20000000;   // x 64 ns sleep: about 1.3 s

// Grid barrier for a cooperative launch (all CTAs resident).  bar[0]:
// arrivals, bar[1]: generation, bar[2]: error word.  Returns false once any
// wait has run out (after `limit` polls).
__device__ bool grid_barrier(unsigned *bar, unsigned nblk, long long limit = kBarrierSpins) {
  __syncthreads();
  if (threadIdx.x == 0) {
    volatile unsigned *gen = bar + 1;
    volatile unsigned *err = bar + 2;
    const unsigned my = *gen;
    __threadfence();
    if (atomicAdd(bar, 1u) == nblk - 1) {
      atomicExch(bar, 0u);
      __threadfence();
      atomicAdd(bar + 1, 1u);
    } else {
      long long spins = 0;
      while (*gen == my && *err == 0u) {
        if (++spins > limit) { atomicExch(bar + 2, 1u); break; }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile unsigned *)(bar + 2) == 0u;
}

// The diagonal leaf's triangular solve L x = w (forward) or L^T x = w
// (backward), m <= 128 rows, L the b x b dense block at L (ld b).  Its lower
// triangle is first staged in shared memory, packed by rows
// (P[r (r + 1) / 2 + c] = L[r, c], c <= r): the whole CTA loads it with
// coalesced reads, then one warp runs the substitution (lanes own rows lane,
// lane + 32, ...) with no global-memory latency in its dependent chain.
__device__ void stage_leaf(const double *__restrict__ L, int b, int m, double *P) {
  for (int e = threadIdx.x; e < m * m; e += blockDim.x) {
    const int r = e % m, c = e / m;
    if (c <= r) P[r * (r + 1) / 2 + c] = L[r + (int64_t)c * b];
  }
}

__device__ void leaf_trsv_packed(const double *P, int m, double *w, bool trans) {
  const int lane = threadIdx.x & 31;
  double x[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) x[q] = (lane + 32 * q < m) ? __ldcg(w + lane + 32 * q) : 0.0;
  for (int s = 0; s < m; ++s) {
    const int i = trans ? m - 1 - s : s;
    const int owner = i & 31, slot = i >> 5;
    double xi = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q)
      if (q == slot) xi = x[q];
    xi = __shfl_sync(0xffffffffu, xi, owner) / P[i * (i + 1) / 2 + i];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int r = lane + 32 * q;
      if (r == i) x[q] = xi;
      else if (r < m && (trans ? r < i : r > i))
        x[q] = fma(-(trans ? P[i * (i + 1) / 2 + r] : P[r * (r + 1) / 2 + i]), xi, x[q]);
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q)
    if (lane + 32 * q < m) w[lane + 32 * q] = x[q];
}

struct SolveArgs {
  FactorArgs F;             // the factor (pools, blocks, panels, ranks)
  const int32_t *diag;      // diagonal block of each leaf
  const int32_t *s0;        // per leaf: range of B tasks (nleaf + 1)
  const int32_t *u0;        // per leaf: range of C rows (nleaf + 1)
  const HTask *hts;         // forward B tasks (right-hand-side panel)
  const UpdRow *rows;       // forward / backward C rows
  const UpdEntry *ents;     // their entries
  const int32_t *bblk;      // backward B tasks: low-rank block ids
  double *w;                // the vector
  double *h;                // coupling vectors: forward at the tasks' own offsets (the
                            // factor's workspace), backward kcap per task of a leaf
  unsigned *bar;
  int nleaf;
  // a batch of nz vectors: vector z and its coupling vectors are w + z zs and
  // h + z hzs, and its factor is F.at(z) (a batch of factors of one tree, or
  // one factor for every vector when F.zstride = 0); every phase runs the
  // tasks of all nz
  int nz;
  int64_t zs, hzs;
};

__global__ void __launch_bounds__(kSolveThreads) k_solve_fwd(SolveArgs S) {
  extern __shared__ double leafP[];   // the packed lower triangle of one diagonal leaf
  const unsigned G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int K = 0; K < S.nleaf; ++K) {
    for (int z = blockIdx.x; z < S.nz; z += G) {
      const FactorArgs F = S.F.at(z);
      const BlockDesc D = F.blocks[S.diag[K]];
      stage_leaf(F.D + D.off_d, F.b, D.rend - D.rbeg, leafP);
      __syncthreads();
      if (warp == 0) leaf_trsv_packed(leafP, D.rend - D.rbeg, S.w + z * S.zs + D.rbeg, false);
      __syncthreads();
    }
    if (!grid_barrier(S.bar, G)) return;
    // B: h_A = W_A^T w[cols A], a warp per component
    const int nb = S.s0[K + 1] - S.s0[K];
    for (int g = blockIdx.x; g < nb * S.nz; g += G) {
      const int z = g / nb, t = S.s0[K] + g % nb;
      const FactorArgs F = S.F.at(z);
      const double *wz = S.w + z * S.zs;
      const HTask T = S.hts[t];
      const BlockDesc A = F.blocks[T.a];
      const PanelDesc PA = F.panels[A.panel];
      const int lda = PA.rend - PA.rbeg, ka = F.rank_l[T.a], p = A.cend - A.cbeg;
      const double *Wa = F.W + PA.off + (int64_t)A.slot * lda + (A.cbeg - PA.rbeg);
      double *h = S.h + z * S.hzs + T.hoff;   // where the sweep's own task writes it
      for (int i = warp; i < ka; i += nw) {
        double s = 0.0;
        for (int k = lane; k < p; k += 32) s = fma(Wa[k + (int64_t)i * lda], __ldcg(wz + A.cbeg + k), s);
        s = warp_sum(s);
        if (lane == 0) h[i] = s;
      }
    }
    if (!grid_barrier(S.bar, G)) return;
    // C: w[I] -= sum over the row's entries, in order
    const int nu = S.u0[K + 1] - S.u0[K];
    for (int g = blockIdx.x; g < nu * S.nz; g += G) {
      const int z = g / nu, t = S.u0[K] + g % nu;
      const FactorArgs F = S.F.at(z);
      double *wz = S.w + z * S.zs;
      const double *hz = S.h + z * S.hzs;
      const UpdRow R = S.rows[t];
      const int I0 = F.leaf_beg[R.leaf], I1 = F.leaf_beg[R.leaf + 1];
      for (int i = I0 + threadIdx.x; i < I1; i += blockDim.x) {
        double acc = 0.0;
        for (int q = R.e0; q < R.e1; ++q) {
          const UpdEntry E = S.ents[q];
          const BlockDesc A = F.blocks[E.a];
          if (E.hoff < 0) {   // dense: D_A w[cols A]
            const double *Dr = F.D + A.off_d + (i - A.rbeg);
            for (int j = 0; j < A.cend - A.cbeg; ++j) acc = fma(Dr[(int64_t)j * F.b], __ldcg(wz + A.cbeg + j), acc);
          } else {            // low rank: U_A[i] h_A (h slot from the task list)
            const double *U = F.U + A.off_u + (i - A.rbeg);
            const int m = A.rend - A.rbeg;
            const double *h = hz + E.hoff;
            for (int k = 0; k < F.rank_l[E.a]; ++k) acc = fma(U[(int64_t)k * m], __ldcg(h + k), acc);
          }
        }
        wz[i] = __ldcg(wz + i) - acc;
      }
    }
    if (!grid_barrier(S.bar, G)) return;
  }
}

__global__ void __launch_bounds__(kSolveThreads) k_solve_bwd(SolveArgs S) {
  extern __shared__ double leafP[];   // the packed lower triangle of one diagonal leaf
  const unsigned G = gridDim.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int K = S.nleaf - 1; K >= 0; --K) {
    for (int z = blockIdx.x; z < S.nz; z += G) {
      const FactorArgs F = S.F.at(z);
      const BlockDesc D = F.blocks[S.diag[K]];
      stage_leaf(F.D + D.off_d, F.b, D.rend - D.rbeg, leafP);
      __syncthreads();
      if (warp == 0) leaf_trsv_packed(leafP, D.rend - D.rbeg, S.w + z * S.zs + D.rbeg, true);
      __syncthreads();
    }
    if (!grid_barrier(S.bar, G)) return;
    // B: h_A = U_A^T v[rows A] for the low-rank blocks whose rows start at K
    const int nb = S.s0[K + 1] - S.s0[K];
    for (int g = blockIdx.x; g < nb * S.nz; g += G) {
      const int z = g / nb, t = S.s0[K] + g % nb;
      const FactorArgs F = S.F.at(z);
      const double *wz = S.w + z * S.zs;
      const int blk = S.bblk[t];
      const BlockDesc A = F.blocks[blk];
      const int m = A.rend - A.rbeg, ka = F.rank_l[blk];
      const double *U = F.U + A.off_u;
      double *h = S.h + z * S.hzs + (int64_t)(t - S.s0[K]) * F.kcap;
      for (int i = warp; i < ka; i += nw) {
        double s = 0.0;
        for (int k = lane; k < m; k += 32) s = fma(U[k + (int64_t)i * m], __ldcg(wz + A.rbeg + k), s);
        s = warp_sum(s);
        if (lane == 0) h[i] = s;
      }
    }
    if (!grid_barrier(S.bar, G)) return;
    // C: v[J] -= sum over the column leaf's entries, in order
    const int nu = S.u0[K + 1] - S.u0[K];
    for (int g = blockIdx.x; g < nu * S.nz; g += G) {
      const int z = g / nu, t = S.u0[K] + g % nu;
      const FactorArgs F = S.F.at(z);
      double *wz = S.w + z * S.zs;
      const double *hz = S.h + z * S.hzs;
      const UpdRow R = S.rows[t];
      const int J0 = F.leaf_beg[R.leaf], J1 = F.leaf_beg[R.leaf + 1];
      for (int j = J0 + threadIdx.x; j < J1; j += blockDim.x) {
        double acc = 0.0;
        for (int q = R.e0; q < R.e1; ++q) {
          const UpdEntry E = S.ents[q];
          const BlockDesc A = F.blocks[E.a];
          if (E.hoff < 0) {   // dense: D_A^T v[rows A], column j - cbeg
            const double *Dc = F.D + A.off_d + (int64_t)(j - A.cbeg) * F.b;
            for (int i = 0; i < A.rend - A.rbeg; ++i) acc = fma(Dc[i], __ldcg(wz + A.rbeg + i), acc);
          } else {            // low rank: W_A[j] h_A
            const PanelDesc PA = F.panels[A.panel];
            const int lda = PA.rend - PA.rbeg;
            const double *Wr = F.W + PA.off + (int64_t)A.slot * lda + (j - PA.rbeg);
            const double *h = hz + E.hoff * F.kcap;
            for (int k = 0; k < F.rank_l[E.a]; ++k) acc = fma(Wr[(int64_t)k * lda], __ldcg(h + k), acc);
          }
        }
        wz[j] = __ldcg(wz + j) - acc;
      }
    }
    if (!grid_barrier(S.bar, G)) return;
  }
}

// failure-detection self-test: one barrier expecting `expect` arrivals
__global__ void k_barrier_selftest(unsigned *bar, unsigned expect, long long limit) {
  grid_barrier(bar, expect, limit);
}

// shared memory of the packed leaf (b (b + 1) / 2 doubles) for leaf size b
int leaf_smem(int b) { return b * (b + 1) / 2 * (int)sizeof(double); }

// the cooperative grid: at most 2 CTAs per SM, as many as fit with smem bytes
// of dynamic shared memory (cached per size)
int solve_grid(int smem = 0) {
  static std::mutex mu;
  std::lock_guard<std::mutex> lk(mu);
  static int cached_smem[4] = {-1, -1, -1, -1}, cached_grid[4] = {0, 0, 0, 0};
  for (int k = 0; k < 4; ++k)
    if (cached_smem[k] == smem) return cached_grid[k];
  int dev = 0, sms = 0, per = 0, per2 = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  cudaFuncSetAttribute(k_solve_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem(kMaxLeaf));
  cudaFuncSetAttribute(k_solve_bwd, cudaFuncAttributeMaxDynamicSharedMemorySize, leaf_smem(kMaxLeaf));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_solve_fwd, kSolveThreads, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k_solve_bwd, kSolveThreads, smem);
  const int g = std::max(1, std::min(std::min(per, per2), 2) * sms);
  for (int k = 0; k < 4; ++k)
    if (cached_smem[k] < 0) { cached_smem[k] = smem; cached_grid[k] = g; break; }
  return g;
}

cudaError_t launch_coop(const void *fn, SolveArgs &S, cudaStream_t st) {
  void *args[] = {&S};
  const int smem = leaf_smem(S.F.b);
  return cudaLaunchCooperativeKernel(fn, dim3(solve_grid(smem)), dim3(kSolveThreads), args, smem, st);
}

}  // namespace

cudaError_t persistent_solve(cudaStream_t st, const FactorArgs &F, const SolvePlan &P, double *w,
                             double *h, unsigned *bar, bool backward) {
  SolveArgs S;
  S.F = F;
  S.diag = P.diag;
  S.nleaf = P.nleaf;
  S.w = w;
  S.h = h;
  S.bar = bar;
  S.nz = F.nz > 0 ? F.nz : 1;
  S.zs = F.zstride / (int64_t)sizeof(double);
  S.hzs = S.zs;
  // arrivals and generation start at zero; the error word is kept (set to
  // zero by the caller once), so a later sweep does not hide an earlier one's
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (!backward) {
    S.s0 = P.ht0; S.u0 = P.ur0; S.hts = P.hts; S.rows = P.urows; S.ents = P.uents; S.bblk = nullptr;
    return launch_coop((const void *)k_solve_fwd, S, st);
  }
  S.s0 = P.bh0; S.u0 = P.bu0; S.hts = nullptr; S.rows = P.bupd; S.ents = P.bents; S.bblk = P.bblk;
  return launch_coop((const void *)k_solve_bwd, S, st);
}

cudaError_t persistent_solve_multi(cudaStream_t st, const FactorArgs &F1, const SolvePlan &P, double *w,
                                   int64_t ws, double *h, int64_t hs, int nrhs, unsigned *bar, bool backward) {
  SolveArgs S;
  S.F = F1;
  S.F.nz = 1;
  S.F.zstride = 0;   // F.at(z) is the one factor for every vector
  S.diag = P.diag;
  S.nleaf = P.nleaf;
  S.w = w;
  S.h = h;
  S.bar = bar;
  S.nz = nrhs;
  S.zs = ws;
  S.hzs = hs;
  cudaError_t e = cudaMemsetAsync(bar, 0, 2 * sizeof(unsigned), st);
  if (e != cudaSuccess) return e;
  if (!backward) {
    S.s0 = P.ht0; S.u0 = P.ur0; S.hts = P.hts; S.rows = P.urows; S.ents = P.uents; S.bblk = nullptr;
    return launch_coop((const void *)k_solve_fwd, S, st);
  }
  S.s0 = P.bh0; S.u0 = P.bu0; S.hts = nullptr; S.rows = P.bupd; S.ents = P.bents; S.bblk = P.bblk;
  return launch_coop((const void *)k_solve_bwd, S, st);
}

}  // namespace hmle

extern "C" __attribute__((visibility("hidden"))) cudaStream_t hmle_internal_ctx_stream(const hmle_ctx *ctx);

extern "C" hmle_status hmle_selftest_barrier(hmle_ctx *ctx, int32_t extra, uint32_t *err_word) {
  using namespace hmle;
  if (!ctx || extra < 0 || extra > 1) return HMLE_ERR_INVALID_ARG;
  cudaStream_t st = hmle_internal_ctx_stream(ctx);
  unsigned *bar = nullptr;
  unsigned h = 0;
  cudaError_t e = cudaMallocAsync(&bar, 3 * sizeof(unsigned), st);
  if (e != cudaSuccess) { cudaGetLastError(); return HMLE_ERR_OOM; }
  e = cudaMemsetAsync(bar, 0, 3 * sizeof(unsigned), st);
  const int G = solve_grid();
  unsigned expect = (unsigned)G + (unsigned)extra;
  long long limit = 2000000;   // about a quarter of a second of polling
  void *args[] = {&bar, &expect, &limit};
  if (e == cudaSuccess)
    e = cudaLaunchCooperativeKernel((const void *)k_barrier_selftest, dim3(G), dim3(kSolveThreads), args, 0, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(&h, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFreeAsync(bar, st);
  cudaStreamSynchronize(st);
  if (e != cudaSuccess) { cudaGetLastError(); return HMLE_ERR_CUDA; }
  if (err_word) *err_word = h;
  return h ? HMLE_ERR_TIMEOUT : HMLE_OK;
}
