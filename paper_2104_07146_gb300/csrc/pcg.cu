// a14 (mixed form): the quadratic form Z^T C~^{-1} Z won back to FP64
// accuracy by preconditioned conjugate gradients.  The operator is the FP64
// H-matrix of C (the assembled dense near-field blocks, admissible blocks as
// their ACA factors U V^T); the preconditioner is the
// H-Cholesky factor of the mixed form, applied as a forward and a backward
// sweep (M^{-1} = L~^{-T} L~^{-1}).  Everything is in cluster order.
//
// All reductions run in a fixed order, so a PCG run is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>

#include "common.cuh"
#include "hmle_internal.h"
#include "kernels.cuh"
#include "matern.cuh"

namespace hmle {
namespace {

constexpr int kDotCtas = 152;   // first-stage CTAs of a dot product (one per SM)
constexpr int kThreadsMv = 128;

// --- y = C x, deterministic ------------------------------------------------
// Stage 1: per admissible block of C, t1 = V^T x[cols], t2 = U^T x[rows].
__global__ void __launch_bounds__(kThreadsMv) k_cmv_t(AsmArgs A, const double *__restrict__ x,
                                                      double *__restrict__ t) {
  __shared__ double red[32];
  const int blk = A.lr_ids[blockIdx.x];
  const BlockDesc B = A.blocks[blk];
  const int m = B.rend - B.rbeg, p = B.cend - B.cbeg, kc = A.kc;
  const int k = A.rank_c[blk];
  const double *U = A.uc + B.off_uc, *V = A.uc + B.off_vc;
  double *t1 = t + (int64_t)blockIdx.x * 2 * kc, *t2 = t1 + kc;
  for (int l = 0; l < k; ++l) {
    double a = 0.0, c = 0.0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) a = fma(V[(int64_t)l * p + j], x[B.cbeg + j], a);
    for (int i = threadIdx.x; i < m; i += blockDim.x) c = fma(U[(int64_t)l * m + i], x[B.rbeg + i], c);
    a = block_sum(a, red);
    c = block_sum(c, red);
    if (threadIdx.x == 0) { t1[l] = a; t2[l] = c; }
  }
}

// Stage 2: one CTA per leaf I; thread i sums, in list order, the blocks whose
// rows cover I (C x[cols], U t1) and then those whose columns cover I
// (C^T x[rows], V t2).  lr_slot[blk]: the block's index among the admissible
// blocks (its t1/t2 slot), -1 for a dense block.
__global__ void __launch_bounds__(kThreadsMv) k_cmv_rows(AsmArgs A, const int32_t *__restrict__ leaf_beg,
                                                         const int32_t *__restrict__ row0,
                                                         const int32_t *__restrict__ rblocks,
                                                         const int32_t *__restrict__ col0,
                                                         const int32_t *__restrict__ cblocks,
                                                         const int32_t *__restrict__ lr_slot,
                                                         const double *__restrict__ x,
                                                         const double *__restrict__ t,
                                                         double *__restrict__ y) {
  const int I = blockIdx.x;
  const int I0 = leaf_beg[I], I1 = leaf_beg[I + 1];
  const int kc = A.kc;
  for (int i = I0 + threadIdx.x; i < I1; i += blockDim.x) {
    double acc = 0.0;
    for (int q = row0[I]; q < row0[I + 1]; ++q) {
      const int blk = rblocks[q];
      const BlockDesc B = A.blocks[blk];
      const int s = lr_slot[blk];
      if (s < 0) {   // dense: row i - rbeg of the stored block
        const double *Cb = A.Cd + B.off_d + (i - B.rbeg);
        for (int j = 0; j < B.cend - B.cbeg; ++j) acc = fma(Cb[(int64_t)j * A.b], x[B.cbeg + j], acc);
      } else {
        const int m = B.rend - B.rbeg, k = A.rank_c[blk];
        const double *U = A.uc + B.off_uc;
        const double *t1 = t + (int64_t)s * 2 * kc;
        for (int l = 0; l < k; ++l) acc = fma(U[(int64_t)l * m + (i - B.rbeg)], t1[l], acc);
      }
    }
    for (int q = col0[I]; q < col0[I + 1]; ++q) {
      const int blk = cblocks[q];
      const BlockDesc B = A.blocks[blk];
      const int s = lr_slot[blk];
      if (s < 0) {   // dense, transposed: column i - cbeg of the stored block
        const double *Cb = A.Cd + B.off_d + (int64_t)(i - B.cbeg) * A.b;
        for (int j = 0; j < B.rend - B.rbeg; ++j) acc = fma(Cb[j], x[B.rbeg + j], acc);
      } else {
        const int p = B.cend - B.cbeg, k = A.rank_c[blk];
        const double *V = A.uc + B.off_vc;
        const double *t2 = t + (int64_t)s * 2 * kc + kc;
        for (int l = 0; l < k; ++l) acc = fma(V[(int64_t)l * p + (i - B.cbeg)], t2[l], acc);
      }
    }
    y[i] = acc;
  }
}

// --- dot products: fixed partition, fixed order -----------------------------
__global__ void k_dot_part(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                           double *__restrict__ part) {
  __shared__ double red[32];
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(a[i], b[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_dot_final(const double *__restrict__ part, int np, double *__restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// --- the scalar recurrences and vector updates ------------------------------
// sc: [0] r.z  [1] p.q  [2] alpha  [3] r.z (new)  [4] beta  [5] r.r  [6] b.b  [7] b.x
__global__ void k_pcg_alpha(double *sc) { sc[2] = sc[0] / sc[1]; }
__global__ void k_pcg_beta(double *sc) {
  sc[4] = sc[3] / sc[0];
  sc[0] = sc[3];
}

__global__ void k_pcg_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                         const double *__restrict__ q, const double *__restrict__ sc, int64_t n) {
  const double alpha = sc[2];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    x[i] = fma(alpha, p[i], x[i]);
    r[i] = fma(-alpha, q[i], r[i]);
  }
}

__global__ void k_pcg_p(double *__restrict__ p, const double *__restrict__ z,
                        const double *__restrict__ sc, int64_t n) {
  const double beta = sc[4];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = fma(beta, p[i], z[i]);
}

void dot(cudaStream_t st, const double *a, const double *b, int64_t n, double *part, double *out) {
  k_dot_part<<<kDotCtas, 256, 0, st>>>(a, b, n, part);
  k_dot_final<<<1, 256, 0, st>>>(part, kDotCtas, out);
}

unsigned grid1(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int64_t pcg_words(int64_t n, int n_lr, int kc, int hmax) {
  return 5 * n + (int64_t)std::max(n_lr, 1) * 2 * kc + (int64_t)hmax + kDotCtas + 16;
}

void launch_cmatvec(cudaStream_t st, const AsmArgs &A, int n_lr, const CmvLists &L,
                    const double *x, double *t, double *y) {
  if (n_lr > 0) k_cmv_t<<<n_lr, kThreadsMv, 0, st>>>(A, x, t);
  k_cmv_rows<<<L.nleaf, kThreadsMv, 0, st>>>(A, L.leaf_beg, L.row0, L.rblocks, L.col0, L.cblocks,
                                             L.lr_slot, x, t, y);
}

namespace {

struct PcgBufs {
  double *x, *r, *z, *p, *qv, *t, *hbuf, *part, *sc;
};

PcgBufs carve(double *pool, int64_t n, int n_lr, int kc, const Plan &PL) {
  PcgBufs B;
  B.x = pool; B.r = B.x + n; B.z = B.r + n; B.p = B.z + n; B.qv = B.p + n;
  B.t = B.qv + n;
  B.hbuf = B.t + (int64_t)std::max(n_lr, 1) * 2 * kc;
  int hmax = 1;
  for (int K = 0; K < PL.nleaf; ++K) hmax = std::max(hmax, PL.bh0[K + 1] - PL.bh0[K]);
  B.part = B.hbuf + (int64_t)hmax * PL.kcap;
  B.sc = B.part + kDotCtas;
  return B;
}

// z = M^{-1} r = L~^{-T} L~^{-1} r through the right-hand-side panel
void precond(cudaStream_t st, const FactorArgs &Fs, const Plan &PL, const int32_t *wpan_rhs,
             const int32_t *bh_blocks, const UpdRow *bupd, const UpdEntry *bents, double *panel,
             const double *r, double *z, double *hbuf, int64_t n, const SolvePlan *SP,
             unsigned *bar) {
  cudaMemcpyAsync(panel, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
  if (SP) {
    persistent_solve(st, Fs, *SP, panel, Fs.ws, bar, false);
    persistent_solve(st, Fs, *SP, panel, hbuf, bar, true);
  } else {
    launch_solve(st, Fs, PL, wpan_rhs);
    launch_backward(st, Fs, PL, panel, bh_blocks, bupd, bents, hbuf);
  }
  cudaMemcpyAsync(z, panel, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
}

// Run seq() directly, or through a graph captured into *g on first use.
template <class Seq>
cudaError_t run_seq(cudaStream_t st, cudaGraphExec_t *g, Seq seq) {
  if (!g) { seq(); return cudaGetLastError(); }
  if (!*g) {
    cudaGraph_t graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { cudaGetLastError(); seq(); return cudaGetLastError(); }
    seq();
    e = cudaStreamEndCapture(st, &graph);
    if (e != cudaSuccess) return e;
    e = cudaGraphInstantiate(g, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) { *g = nullptr; return e; }
  }
  return cudaGraphLaunch(*g, st);
}

}  // namespace

namespace {

cudaError_t launch_iteration(PcgRun &R) {
  const PcgBufs B = carve(R.pool, R.n, R.n_lr, R.A.kc, *R.PL);
  cudaStream_t st = R.st;
  const int64_t n = R.n;
  // one iteration; the preconditioner of the next one runs even when this
  // one converges (its result is then unused)
  cudaError_t e = run_seq(st, R.g_iter, [&] {
    launch_cmatvec(st, R.A, R.n_lr, R.L, B.p, B.t, B.qv);
    dot(st, B.p, B.qv, n, B.part, B.sc + 1);
    k_pcg_alpha<<<1, 1, 0, st>>>(B.sc);
    k_pcg_xr<<<grid1(n), 256, 0, st>>>(B.x, B.r, B.p, B.qv, B.sc, n);
    dot(st, B.r, B.r, n, B.part, B.sc + 5);
    precond(st, R.Fs, *R.PL, R.wpan_rhs, R.bh_blocks, R.bupd, R.bents, R.panel, B.r, B.z, B.hbuf, n,
            R.SP, R.bar);
    dot(st, B.r, B.z, n, B.part, B.sc + 3);
    k_pcg_beta<<<1, 1, 0, st>>>(B.sc);
    k_pcg_p<<<grid1(n), 256, 0, st>>>(B.p, B.z, B.sc, n);
  });
  if (e != cudaSuccess) return e;
  if (R.SP) {
    e = cudaMemcpyAsync(reinterpret_cast<unsigned *>(R.host + 3), R.bar + 2, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
  }
  return cudaMemcpyAsync(R.host + 1, B.sc + 5, sizeof(double), cudaMemcpyDeviceToHost, st);
}

// Eq. 4 (kriging): out[j] = sum_i sigma2 M_nu(|s2_j - s1_i| / ell) x_i, one
// CTA per new location, the training points (SoA, cluster order) read in
// order and the partial sums reduced in a fixed order.  No nugget: the new
// locations are other points than the training ones.
__global__ void k_cross_matvec(const double *__restrict__ tab, const double *__restrict__ xyz,
                               int64_t n, int d, const double *__restrict__ locs2, double inv_ell,
                               double sigma2, const double *__restrict__ x, double *__restrict__ out) {
  __shared__ double red[32];
  const int64_t j = blockIdx.x;
  double p[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < d; ++k) p[k] = locs2[j * d + k];
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    double h2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double dx = p[k] - xyz[k * n + i];
      h2 = fma(dx, dx, h2);
    }
    acc = fma(sigma2 * matern_unit(tab, sqrt(h2) * inv_ell), x[i], acc);
  }
  acc = block_sum(acc, red);
  if (threadIdx.x == 0) out[j] = acc;
}

}  // namespace

// The transposed product: out[i] = sum_j sigma2 M_nu(|s1_i - s2_j| / ell) y_j,
// one thread per training point (cluster order), the m new locations summed
// in order.
__global__ void k_cross_matvec_t(const double *__restrict__ tab, const double *__restrict__ xyz,
                                 int64_t n, int d, const double *__restrict__ locs2, int64_t m,
                                 double inv_ell, double sigma2, const double *__restrict__ y,
                                 double *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double p[3] = {0.0, 0.0, 0.0};
  for (int k = 0; k < d; ++k) p[k] = xyz[k * n + i];
  double acc = 0.0;
  for (int64_t j = 0; j < m; ++j) {
    double h2 = 0.0;
    for (int k = 0; k < d; ++k) {
      const double dx = p[k] - locs2[j * d + k];
      h2 = fma(dx, dx, h2);
    }
    acc = fma(sigma2 * matern_unit(tab, sqrt(h2) * inv_ell), y[j], acc);
  }
  out[i] = acc;
}

void launch_cross_matvec(cudaStream_t st, const double *tab, const double *xyz, int64_t n, int d,
                         const double *locs2, int64_t m, double inv_ell, double sigma2,
                         const double *x, double *out) {
  if (m > 0) k_cross_matvec<<<(unsigned)m, 256, 0, st>>>(tab, xyz, n, d, locs2, inv_ell, sigma2, x, out);
}

void launch_cross_matvec_t(cudaStream_t st, const double *tab, const double *xyz, int64_t n, int d,
                           const double *locs2, int64_t m, double inv_ell, double sigma2,
                           const double *y, double *out) {
  if (n > 0)
    k_cross_matvec_t<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(tab, xyz, n, d, locs2, m, inv_ell,
                                                                 sigma2, y, out);
}

cudaError_t pcg_start(PcgRun &R) {
  const PcgBufs B = carve(R.pool, R.n, R.n_lr, R.A.kc, *R.PL);
  cudaStream_t st = R.st;
  const int64_t n = R.n;
  R.it = 0;
  R.rel = 1.0;
  R.state = 0;
  R.timed_out = false;
  *reinterpret_cast<unsigned *>(R.host + 3) = 0u;
  if (R.SP) {
    cudaError_t e0 = cudaMemsetAsync(R.bar, 0, 3 * sizeof(unsigned), st);
    if (e0 != cudaSuccess) return e0;
  }
  // x = 0, r = b, z = M^{-1} r, p = z, sc[0] = r.z, sc[6] = b.b
  cudaError_t e = run_seq(st, R.g_init, [&] {
    cudaMemsetAsync(B.x, 0, sizeof(double) * n, st);
    cudaMemcpyAsync(B.r, R.b, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    precond(st, R.Fs, *R.PL, R.wpan_rhs, R.bh_blocks, R.bupd, R.bents, R.panel, B.r, B.z, B.hbuf, n,
            R.SP, R.bar);
    cudaMemcpyAsync(B.p, B.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, st);
    dot(st, B.r, B.z, n, B.part, B.sc + 0);
    dot(st, R.b, R.b, n, B.part, B.sc + 6);
  });
  if (e == cudaSuccess) e = cudaMemcpyAsync(R.host + 0, B.sc + 6, sizeof(double), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && R.maxit > 0) e = launch_iteration(R);
  return e;
}

cudaError_t pcg_poll(PcgRun &R, bool *finished) {
  *finished = false;
  if (R.state == 2) { *finished = true; return cudaSuccess; }
  const PcgBufs B = carve(R.pool, R.n, R.n_lr, R.A.kc, *R.PL);
  if (R.state == 1) {   // the final dot has completed
    R.q = R.host[2];
    R.state = 2;
    *finished = true;
    return cudaGetLastError();
  }
  if (R.SP && *reinterpret_cast<volatile unsigned *>(R.host + 3) != 0u) {
    R.timed_out = true;   // a persistent sweep gave up at a barrier: stop here
    R.state = 2;
    *finished = true;
    return cudaSuccess;
  }
  if (R.maxit > 0) {    // an iteration has completed
    ++R.it;
    const double bb = R.host[0];
    R.rel = bb > 0.0 ? std::sqrt(R.host[1] / bb) : 0.0;
  }
  if (R.it < R.maxit && R.rel > R.tol) return launch_iteration(R);
  // converged, out of iterations or not finite: q = b.x
  dot(R.st, R.b, B.x, R.n, B.part, B.sc + 7);
  R.state = 1;
  return cudaMemcpyAsync(R.host + 2, B.sc + 7, sizeof(double), cudaMemcpyDeviceToHost, R.st);
}

cudaError_t pcg_quad(PcgRun &R) {
  cudaError_t e = pcg_start(R);
  bool fin = false;
  while (e == cudaSuccess && !fin) {
    e = cudaStreamSynchronize(R.st);
    if (e == cudaSuccess) e = pcg_poll(R, &fin);
  }
  return e;
}

}  // namespace hmle
