// a3-a4 (Eq. 2; Sec. 2): assembly of the H-matrix C~(theta) on the device.
//
//  * k_matern_table: Chebyshev tables of M_nu for this theta (matern.cuh).
//  * k_aca: adaptive cross approximation of every admissible block
//    C_{rho,sigma} ~= U V^T, generated from single rows and columns of the
//    kernel (partial pivoting: the next row pivot is the largest entry of the
//    last column outside the rows already used).  Stops when
//    |u_k| |v_k| <= eps |S_k|_F, with |S_k|_F^2 updated from the new cross
//    and its inner products with the previous ones.
//  * k_assemble_dense: the dense near-field blocks of C, stored per theta
//    (read by the factorisation's dense targets and by the H-matvec).
#include <cuda_runtime.h>

#include "common.cuh"
#include "hmle_internal.h"
#include "kernels.cuh"
#include "matern.cuh"

namespace hmle {

// One block per interval; thread k computes node k.
__global__ void k_matern_table(double nu, double *__restrict__ tab) {
  __shared__ double f[kNcoef];
  const int j = blockIdx.x;
  const double lognorm = (nu - 1.0) * log(2.0) + lgamma(nu);
  if (j == 0 && threadIdx.x == 0) {
    tab[0] = nu;
    tab[1] = lognorm;
    for (int q = 2; q < 8; ++q) tab[q] = 0.0;
  }
  const double a = ldexp(1.0, kJmin + j);
  const double pi = 3.141592653589793238462643383279502884;
  for (int k = threadIdx.x; k < kNcoef; k += blockDim.x) {
    double tk = cos(pi * (k + 0.5) / kNcoef);
    double x = a * (tk + 3.0) * 0.5;
    f[k] = matern_unit_quad(nu, lognorm, x);
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kNcoef; c += blockDim.x) {
    double s = 0.0;
    for (int k = 0; k < kNcoef; ++k) s += f[k] * cos(pi * c * (k + 0.5) / kNcoef);
    s *= 2.0 / kNcoef;
    if (c == 0) s *= 0.5;
    tab[8 + j * kNcoef + c] = s;
  }
}

// Evaluate M_nu at m points through the table (check of the device Bessel path).
__global__ void k_matern_eval(const double *__restrict__ tab, const double *__restrict__ x,
                              int64_t m, double *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = matern_unit(tab, x[i]);
}

// ACA of admissible block blk_ids[blockIdx.x].
__global__ void __launch_bounds__(256) k_aca(AsmArgs A) {
  __shared__ double redv[32];
  __shared__ int redi[32];
  __shared__ double dots_u[kMaxRank + 8];
  __shared__ double dots_v[kMaxRank + 8];
  __shared__ int used[kMaxRank + 8];
  __shared__ int s_istar;
  const int blk = A.lr_ids[blockIdx.x];
  const BlockDesc B = A.blocks[blk];
  const int m = B.rend - B.rbeg, p = B.cend - B.cbeg;
  const int kc = A.kc;
  double *U = A.uc + B.off_uc;   // m x kc, ld m
  double *V = A.uc + B.off_vc;   // p x kc, ld p
  const double inv_ell = A.inv_ell, s2 = A.sigma2;
  int istar = 0, nused = 0, rank = 0;
  double norm2 = 0.0;
  bool done = false, overflow = false;
  int tries = 0;
  for (int k = 0; k < kc && !done; ) {
    // row istar of the residual: v_j = C(r, c_j) - sum_l U[r,l] V[j,l]
    const int64_t gi = B.rbeg + istar;
    double best = 0.0;
    int bidx = 0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      double v = cov_entry(A.tab, A.xyz, A.n, A.d, gi, B.cbeg + j, inv_ell, s2, 0.0);
      for (int l = 0; l < k; ++l) v = fma(-U[(int64_t)l * m + istar], V[(int64_t)l * p + j], v);
      V[(int64_t)k * p + j] = v;
      if (fabs(v) > fabs(best)) { best = v; bidx = j; }
    }
    double pv;
    int jstar;
    block_argmax_abs(best, bidx, redv, redi, &pv, &jstar);
    if (threadIdx.x == 0) used[nused] = istar;
    ++nused;
    if (pv == 0.0 || !isfinite(pv)) {
      // this row is already represented; try the next unused row
      if (++tries > 3 || nused >= kc + 4) { done = true; break; }
      __syncthreads();
      if (threadIdx.x == 0) {
        int r = istar;
        for (int q = 0; q < m; ++q) {
          r = (r + 1) % m;
          bool u = false;
          for (int w = 0; w < nused; ++w) u |= (used[w] == r);
          if (!u) break;
        }
        s_istar = r;
      }
      __syncthreads();
      istar = s_istar;
      continue;
    }
    const double inv = 1.0 / pv;
    for (int j = threadIdx.x; j < p; j += blockDim.x) V[(int64_t)k * p + j] *= inv;
    __syncthreads();
    // column jstar of the residual
    const int64_t gj = B.cbeg + jstar;
    double bu = 0.0;
    int bui = 0;
    double uu = 0.0;
    for (int i = threadIdx.x; i < m; i += blockDim.x) {
      double u = cov_entry(A.tab, A.xyz, A.n, A.d, B.rbeg + i, gj, inv_ell, s2, 0.0);
      for (int l = 0; l < k; ++l) u = fma(-U[(int64_t)l * m + i], V[(int64_t)l * p + jstar], u);
      U[(int64_t)k * m + i] = u;
      uu = fma(u, u, uu);
      bool isused = false;
      for (int w = 0; w < nused; ++w) isused |= (used[w] == i);
      if (!isused && fabs(u) > fabs(bu)) { bu = u; bui = i; }
    }
    uu = block_sum(uu, redv);
    double vv = 0.0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) {
      double v = V[(int64_t)k * p + j];
      vv = fma(v, v, vv);
    }
    vv = block_sum(vv, redv);
    // inner products with previous crosses
    for (int l = 0; l < k; ++l) {
      double du = 0.0, dv = 0.0;
      for (int i = threadIdx.x; i < m; i += blockDim.x)
        du = fma(U[(int64_t)k * m + i], U[(int64_t)l * m + i], du);
      for (int j = threadIdx.x; j < p; j += blockDim.x)
        dv = fma(V[(int64_t)k * p + j], V[(int64_t)l * p + j], dv);
      du = block_sum(du, redv);
      dv = block_sum(dv, redv);
      if (threadIdx.x == 0) { dots_u[l] = du; dots_v[l] = dv; }
    }
    __syncthreads();
    double cross = 0.0;
    for (int l = 0; l < k; ++l) cross += dots_u[l] * dots_v[l];
    norm2 += 2.0 * cross + uu * vv;
    double pu;
    int inext;
    block_argmax_abs(bu, bui, redv, redi, &pu, &inext);
    ++k;
    rank = k;
    tries = 0;
    if (sqrt(uu * vv) <= A.eps * sqrt(fabs(norm2))) { done = true; break; }
    if (A.fixed_k > 0 && k >= A.fixed_k) { done = true; break; }   // fixed-rank mode
    if (k == kc) { overflow = true; break; }
    istar = inext;
    if (pu == 0.0) {
      // every remaining row is numerically zero in this column: pick the
      // next unused row to keep exploring
      if (threadIdx.x == 0) {
        int r = istar;
        for (int q = 0; q < m; ++q) {
          r = (r + 1) % m;
          bool u = false;
          for (int w = 0; w < nused; ++w) u |= (used[w] == r);
          if (!u) break;
        }
        s_istar = r;
      }
      __syncthreads();
      istar = s_istar;
    }
    if (nused >= m) { done = true; break; }
  }
  // zero the unused columns
  for (int l = rank; l < kc; ++l) {
    for (int i = threadIdx.x; i < m; i += blockDim.x) U[(int64_t)l * m + i] = 0.0;
    for (int j = threadIdx.x; j < p; j += blockDim.x) V[(int64_t)l * p + j] = 0.0;
  }
  if (threadIdx.x == 0) {
    A.rank_c[blk] = rank;
    A.cnorm[blk] = sqrt(fabs(norm2));
    if (overflow) raise_flag(A.flags, kFlagRankOverflow);
  }
}

void launch_matern_table(cudaStream_t st, double nu, double *tab) {
  k_matern_table<<<kNint, 32, 0, st>>>(nu, tab);
}
void launch_matern_eval(cudaStream_t st, const double *tab, const double *x, int64_t m,
                        double *out) {
  if (m > 0) k_matern_eval<<<(unsigned)((m + 255) / 256), 256, 0, st>>>(tab, x, m, out);
}
void launch_aca(cudaStream_t st, const AsmArgs &A, int n_lr) {
  if (n_lr > 0) k_aca<<<n_lr, 256, 0, st>>>(A);
}

// a3: the dense near field.  One CTA per dense block (all leaf-level blocks
// of the lower triangle kept dense, the diagonal ones included, both
// triangles of those): C(i, j) = sigma^2 M_nu(|s_i - s_j| / ell) + tau^2 [i == j]
// into the block's b x b slot (ld b, column-major: consecutive threads write
// consecutive rows), padding rows and columns zero.
__global__ void k_assemble_dense(AsmArgs A, const int32_t *__restrict__ dense_ids, int b,
                                 double *__restrict__ Cd) {
  const BlockDesc B = A.blocks[dense_ids[blockIdx.x]];
  const int m = B.rend - B.rbeg, p = B.cend - B.cbeg;
  double *out = Cd + B.off_d;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    const int i = e % b, j = e / b;
    out[e] = (i < m && j < p) ? cov_entry(A.tab, A.xyz, A.n, A.d, B.rbeg + i, B.cbeg + j, A.inv_ell,
                                          A.sigma2, A.tau2)
                              : 0.0;
  }
}

void launch_assemble_dense(cudaStream_t st, const AsmArgs &A, const int32_t *dense_ids, int nd,
                           int b, double *Cd) {
  if (nd > 0) k_assemble_dense<<<nd, 256, 0, st>>>(A, dense_ids, b, Cd);
}

}  // namespace hmle
