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
// In every kernel below, blockIdx.y selects the evaluation of a batch (its
// vectors at z zs doubles, its H-matrix through AsmArgs::at); one
// evaluation is the batch of one.
__global__ void __launch_bounds__(kThreadsMv) k_cmv_t(AsmArgs Az, const double *__restrict__ x,
                                                      double *__restrict__ t, int64_t zs, int64_t tzs) {
  __shared__ double red[32];
  const AsmArgs A = Az.at(blockIdx.y);
  x += blockIdx.y * zs;
  t += blockIdx.y * tzs;
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
__global__ void __launch_bounds__(kThreadsMv) k_cmv_rows(AsmArgs Az, const int32_t *__restrict__ leaf_beg,
                                                         const int32_t *__restrict__ row0,
                                                         const int32_t *__restrict__ rblocks,
                                                         const int32_t *__restrict__ col0,
                                                         const int32_t *__restrict__ cblocks,
                                                         const int32_t *__restrict__ lr_slot,
                                                         const double *__restrict__ x,
                                                         const double *__restrict__ t,
                                                         double *__restrict__ y, int64_t zs, int64_t tzs) {
  const AsmArgs A = Az.at(blockIdx.y);
  x += blockIdx.y * zs;
  t += blockIdx.y * tzs;
  y += blockIdx.y * zs;
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
                           double *__restrict__ part, int64_t zs) {
  __shared__ double red[32];
  a += blockIdx.y * zs;
  b += blockIdx.y * zs;
  part += blockIdx.y * zs;
  const int64_t chunk = (n + gridDim.x - 1) / gridDim.x;
  const int64_t i0 = blockIdx.x * chunk, i1 = min(n, i0 + chunk);
  double s = 0.0;
  for (int64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) s = fma(a[i], b[i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void k_dot_final(const double *__restrict__ part, int np, double *__restrict__ out, int64_t zs) {
  __shared__ double red[32];
  part += blockIdx.x * zs;
  out += blockIdx.x * zs;
  double s = 0.0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) s += part[i];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = s;
}

// --- the scalar recurrences and vector updates ------------------------------
// sc: [0] r.z  [1] p.q  [2] alpha  [3] r.z (new)  [4] beta  [5] r.r  [6] b.b  [7] b.x
//     [8] stopped (batch)  [9] iterations (batch)  [10] relative residual (batch)
// One thread per evaluation (grid nz).
__global__ void k_pcg_alpha(double *sc, int64_t zs) {
  sc += blockIdx.x * zs;
  sc[2] = sc[0] / sc[1];
}
__global__ void k_pcg_beta(double *sc, int64_t zs) {
  sc += blockIdx.x * zs;
  sc[4] = sc[3] / sc[0];
  sc[0] = sc[3];
}

// x += alpha p, r -= alpha q; an evaluation of a batch that has stopped keeps
// its x (and r) as they were when it stopped.
__global__ void k_pcg_xr(double *__restrict__ x, double *__restrict__ r, const double *__restrict__ p,
                         const double *__restrict__ q, const double *__restrict__ sc, int64_t n, int64_t zs) {
  const int64_t o = blockIdx.y * zs;
  if (sc[o + 8] != 0.0) return;
  const double alpha = sc[o + 2];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) {
    x[o + i] = fma(alpha, p[o + i], x[o + i]);
    r[o + i] = fma(-alpha, q[o + i], r[o + i]);
  }
}

__global__ void k_pcg_p(double *__restrict__ p, const double *__restrict__ z,
                        const double *__restrict__ sc, int64_t n, int64_t zs) {
  const int64_t o = blockIdx.y * zs;
  const double beta = sc[o + 4];
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[o + i] = fma(beta, p[o + i], z[o + i]);
}

// batch: after an iteration's r.r, an evaluation that has not stopped counts
// the iteration and stops where a single solve would (residual at or below
// tol, or maxit iterations, or not finite)
__global__ void k_pcg_check(double *sc, double tol, int maxit, int64_t zs) {
  sc += blockIdx.x * zs;
  if (sc[8] != 0.0) return;
  const double it = sc[9] + 1.0;
  const double bb = sc[6];
  const double rel = bb > 0.0 ? sqrt(sc[5] / bb) : 0.0;
  sc[9] = it;
  sc[10] = rel;
  if (!(it < (double)maxit && rel > tol)) sc[8] = 1.0;
}

__global__ void k_pcg_reset(double *sc, int64_t zs) {
  sc += blockIdx.x * zs;
  sc[8] = 0.0;
  sc[9] = 0.0;
  sc[10] = 1.0;
}

void dot(cudaStream_t st, const double *a, const double *b, int64_t n, double *part, double *out,
         int nz = 1, int64_t zs = 0) {
  k_dot_part<<<dim3(kDotCtas, nz), 256, 0, st>>>(a, b, n, part, zs);
  k_dot_final<<<nz, 256, 0, st>>>(part, kDotCtas, out, zs);
}

unsigned grid1(int64_t n) { return (unsigned)((n + 255) / 256); }

}  // namespace

int64_t pcg_words(int64_t n, int n_lr, int kc, int hmax) {
  return 5 * n + (int64_t)std::max(n_lr, 1) * 2 * kc + (int64_t)hmax + kDotCtas + 16;
}

void launch_cmatvec(cudaStream_t st, const AsmArgs &A, int n_lr, const CmvLists &L,
                    const double *x, double *t, double *y, int nz, int64_t zs, int64_t tzs) {
  if (tzs < 0) tzs = zs;
  if (n_lr > 0) k_cmv_t<<<dim3(n_lr, nz), kThreadsMv, 0, st>>>(A, x, t, zs, tzs);
  k_cmv_rows<<<dim3(L.nleaf, nz), kThreadsMv, 0, st>>>(A, L.leaf_beg, L.row0, L.rblocks, L.col0, L.cblocks,
                                                       L.lr_slot, x, t, y, zs, tzs);
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
void copy_z(cudaStream_t st, double *dst, const double *src, int64_t n, int nz, int64_t zs) {
  cudaMemcpy2DAsync(dst, sizeof(double) * std::max<int64_t>(zs, n), src, sizeof(double) * std::max<int64_t>(zs, n),
                    sizeof(double) * n, nz, cudaMemcpyDeviceToDevice, st);
}

void precond(cudaStream_t st, const FactorArgs &Fs, const Plan &PL, const int32_t *wpan_rhs,
             const int32_t *bh_blocks, const UpdRow *bupd, const UpdEntry *bents, double *panel,
             const double *r, double *z, double *hbuf, int64_t n, const SolvePlan *SP,
             unsigned *bar) {
  const int nz = Fs.nz > 0 ? Fs.nz : 1;
  const int64_t zs = Fs.zstride / (int64_t)sizeof(double);
  copy_z(st, panel, r, n, nz, zs);
  if (SP) {
    persistent_solve(st, Fs, *SP, panel, Fs.ws, bar, false);
    persistent_solve(st, Fs, *SP, panel, hbuf, bar, true);
  } else {
    launch_solve(st, Fs, PL, wpan_rhs);
    launch_backward(st, Fs, PL, panel, bh_blocks, bupd, bents, hbuf);
  }
  copy_z(st, z, panel, n, nz, zs);
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
  const int nz = R.nz;
  const int64_t zs = R.zs;
  cudaError_t e = run_seq(st, R.g_iter, [&] {
    launch_cmatvec(st, R.A, R.n_lr, R.L, B.p, B.t, B.qv, nz, zs);
    dot(st, B.p, B.qv, n, B.part, B.sc + 1, nz, zs);
    k_pcg_alpha<<<nz, 1, 0, st>>>(B.sc, zs);
    k_pcg_xr<<<dim3(grid1(n), nz), 256, 0, st>>>(B.x, B.r, B.p, B.qv, B.sc, n, zs);
    dot(st, B.r, B.r, n, B.part, B.sc + 5, nz, zs);
    if (nz > 1 || R.hostz) k_pcg_check<<<nz, 1, 0, st>>>(B.sc, R.tol, R.maxit, zs);
    precond(st, R.Fs, *R.PL, R.wpan_rhs, R.bh_blocks, R.bupd, R.bents, R.panel, B.r, B.z, B.hbuf, n,
            R.SP, R.bar);
    dot(st, B.r, B.z, n, B.part, B.sc + 3, nz, zs);
    k_pcg_beta<<<nz, 1, 0, st>>>(B.sc, zs);
    k_pcg_p<<<dim3(grid1(n), nz), 256, 0, st>>>(B.p, B.z, B.sc, n, zs);
  });
  if (e != cudaSuccess) return e;
  if (R.SP) {
    e = cudaMemcpyAsync(reinterpret_cast<unsigned *>(R.host + 3), R.bar + 2, sizeof(unsigned),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return e;
  }
  if (R.hostz)   // batch: every evaluation's stop flag, iterations and residual
    return cudaMemcpy2DAsync(R.hostz, 4 * sizeof(double), B.sc + 8, sizeof(double) * zs, 3 * sizeof(double),
                             nz, cudaMemcpyDeviceToHost, st);
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

// Eq. 5-6: columns of C12 for a block of new locations, one thread per
// (training point, column); the training points in cluster order.
__global__ void k_cross_cols(const double *__restrict__ tab, const double *__restrict__ xyz, int64_t n,
                             int d, const double *__restrict__ locs2, int64_t j0, double inv_ell,
                             double sigma2, double *__restrict__ out, int64_t ld) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int jj = blockIdx.y;
  if (i >= n) return;
  const double *p = locs2 + (j0 + jj) * d;
  double h2 = 0.0;
  for (int k = 0; k < d; ++k) {
    const double dx = xyz[k * n + i] - p[k];
    h2 = fma(dx, dx, h2);
  }
  out[i + jj * ld] = sigma2 * matern_unit(tab, sqrt(h2) * inv_ell);
}

// Per-column dot products, one CTA per column, a fixed order of the sums.
__global__ void k_col_dots(const double *__restrict__ a, const double *__restrict__ b, int64_t n,
                           int64_t ld, double *__restrict__ out) {
  __shared__ double red[32];
  const int64_t o = (int64_t)blockIdx.x * ld;
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) s = fma(a[o + i], b[o + i], s);
  s = block_sum(s, red);
  if (threadIdx.x == 0) out[blockIdx.x] = s;
}

void launch_cross_cols(cudaStream_t st, const double *tab, const double *xyz, int64_t n, int d,
                       const double *locs2, int64_t j0, int cnt, double inv_ell, double sigma2, double *out,
                       int64_t ld) {
  if (n > 0 && cnt > 0)
    k_cross_cols<<<dim3((unsigned)((n + 255) / 256), (unsigned)cnt), 256, 0, st>>>(tab, xyz, n, d, locs2, j0,
                                                                                inv_ell, sigma2, out, ld);
}

void launch_col_dots(cudaStream_t st, const double *a, const double *b, int64_t n, int64_t ld, int cnt,
                     double *out) {
  if (cnt > 0) k_col_dots<<<(unsigned)cnt, 256, 0, st>>>(a, b, n, ld, out);
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
  const int nz = R.nz;
  const int64_t zs = R.zs;
  cudaError_t e = run_seq(st, R.g_init, [&] {
    cudaMemset2DAsync(B.x, sizeof(double) * std::max<int64_t>(zs, n), 0, sizeof(double) * n, nz, st);
    copy_z(st, B.r, R.b, n, nz, zs);
    precond(st, R.Fs, *R.PL, R.wpan_rhs, R.bh_blocks, R.bupd, R.bents, R.panel, B.r, B.z, B.hbuf, n,
            R.SP, R.bar);
    copy_z(st, B.p, B.z, n, nz, zs);
    dot(st, B.r, B.z, n, B.part, B.sc + 0, nz, zs);
    dot(st, R.b, R.b, n, B.part, B.sc + 6, nz, zs);
    k_pcg_reset<<<nz, 1, 0, st>>>(B.sc, zs);
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

// A batch of R.nz solves in lockstep: one launch per kernel for all of them
// (the persistent sweeps included); each evaluation stops updating its
// solution where its single solve would stop, and the batch iterates until
// every evaluation has stopped.  The host reads the nz stop flags after each
// iteration.
cudaError_t pcg_batch_start(PcgRun &R) {
  R.it = 0;
  R.state = 0;
  R.timed_out = false;
  R.itz.assign(R.nz, 0);
  R.relz.assign(R.nz, 1.0);
  R.qz.assign(R.nz, 0.0);
  return pcg_start(R);   // the set-up, then the first iteration (nz-aware)
}

cudaError_t pcg_batch_poll(PcgRun &R, bool *finished) {
  *finished = false;
  const PcgBufs B = carve(R.pool, R.n, R.n_lr, R.A.kc, *R.PL);
  if (R.state == 2) { *finished = true; return cudaSuccess; }
  if (R.state == 1) {   // the final dots have completed
    for (int z = 0; z < R.nz; ++z) R.qz[z] = R.hostz[4 * z + 3];
    R.state = 2;
    *finished = true;
    return cudaGetLastError();
  }
  if (R.SP && *reinterpret_cast<volatile unsigned *>(R.host + 3) != 0u) {
    R.timed_out = true;
    R.state = 2;
    *finished = true;
    return cudaSuccess;
  }
  bool all = true;
  for (int z = 0; z < R.nz; ++z) {
    R.itz[z] = (int)R.hostz[4 * z + 1];
    R.relz[z] = R.hostz[4 * z + 2];
    all = all && (R.maxit <= 0 || R.hostz[4 * z] != 0.0);
  }
  ++R.it;
  if (!all && R.it < R.maxit) return launch_iteration(R);
  // every evaluation has stopped: q = b.x
  dot(R.st, R.b, B.x, R.n, B.part, B.sc + 7, R.nz, R.zs);
  R.state = 1;
  return cudaMemcpy2DAsync(R.hostz + 3, 4 * sizeof(double), B.sc + 7, sizeof(double) * R.zs, sizeof(double),
                           R.nz, cudaMemcpyDeviceToHost, R.st);
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
