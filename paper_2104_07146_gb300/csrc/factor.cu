// a6-a11 (Sec. 2): the left-looking leaf sweep of the H-Cholesky
// factorisation C~ = L~ L~^T with the forward solve w = L~^{-1} P Z fused in.
//
// One step K runs these phases (the planner fixes every task list):
//  P1  k_gram        G_AB = W_A[ov]^T W_B[ov] for pairs of low-rank blocks.
//  P2  k_side_t/s, k_rows   Y = S_T Omega for every low-rank target T whose
//      column cluster starts at K, with S_T = C_T - sum_pairs U_A G_AB U_B^T
//      and Omega a counter-based random sign matrix.
//  P3  k_tsqr_part, k_tsqr_final, k_tall_apply, k_cholqr_part/final,
//      k_tall_apply   Q = orth(Y): the R factor of Y by Householder
//      reflections over row groups (TSQR), a column-pivoted QR of that R
//      (R P = Q_r R_p, stopped where the pivot norm falls below 1e-14 of the
//      first), Q1 = Y P R_p11^{-1}, then one CholQR pass that restores
//      orthogonality to rounding level.
//  P4  as P2 with S_T^T applied to Q: Z = S_T^T Q.
//  P5  k_tsqr_part, k_tsqr_final (truncating), k_tall_apply   the SVD of Z
//      from its R factor (pivoted QR, then one-sided Jacobi on R_p^T); keep
//      the leading k with tail energy sum_{i>=k} sigma_i^2 <= eps^2
//      max(|S_T|_F^2, |C_T|_F^2) (or the leading fixed_k in the fixed-rank
//      mode): U_T = Q V_k, W_T = Z V_k (the start of the forward solve of W_T).
//  P6  k_dense_pair, k_dense_reduce   S_IK = C_IK - sum_pairs U_A G_AB U_B^T for the dense
//      blocks of column K (diagonal first); C_IK from the assembled dense
//      near field.
//  P7  k_potrf       L_KK = chol(S_KK); log-det part 2 sum log L_ii.
//  P8  k_trsm        L_IK = S_IK L_KK^{-T}.
//  P9  k_wsolve      rows of leaf K of every open W-panel: W <- L_KK^{-1} W.
//  P10 k_htask, k_updrow   blocks A whose columns end at K push
//      W[rows A] -= U_A (W_A^T W[cols A]) (dense A: D_A W[cols A]) into every
//      open panel containing them.
// All FP64, except that the mixed form runs the update products (k_gram,
// k_side_t/s, k_rows, k_dense_pair, k_htask, k_updrow) in FP32 (template
// parameter Tc).  Every output element is written by exactly one thread, in
// a fixed order: the sweep is deterministic.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>

#include "common.cuh"
#include "hmle_internal.h"
#include "kernels.cuh"
#include "matern.cuh"
#include "tc_gemm.cuh"

namespace hmle {

namespace {

constexpr int kThreads = 128;
constexpr int kMaxEntries = 512;     // side entries covering one leaf row of a target
constexpr int kMaxRowK = 8192;       // concatenated columns of one row task
constexpr int kTM = 64, kTN = 64, kTK = 16;
constexpr int kGemmSmem = kTK * (kTM + kTN);  // doubles

// C(i, j) = sum_k A(i, k) B(k, j) for i < M, j < N, k < K, delivered to
// fc(i, j, value).  A_KFAST / B_KFAST: the operand is contiguous along k in
// memory (chooses the coalesced loading order).  128 threads, 64 x TNX
// output tiles (TNX = 64 or 32), 4 x (TNX / 8) register micro-tiles, K
// staged 16 at a time, the next 16 read into registers while the current
// ones are multiplied.  T: the arithmetic type (double): operands are
// rounded to T as they are staged, products accumulate in T, and fc receives
// the sum as a double.
template <class T, bool A_KFAST, bool B_KFAST, int TNX, class FA, class FB, class FC>
__device__ void cta_gemm_t(int M, int N, int K, FA fa, FB fb, FC fc, double *smem) {
  constexpr int MC = TNX / 8;
  T *sA = reinterpret_cast<T *>(smem);
  T *sB = sA + kTK * kTM;
  const int tid = threadIdx.x;
  const int ti = tid & 15, tj = tid >> 4;
  for (int i0 = 0; i0 < M; i0 += kTM) {
    for (int j0 = 0; j0 < N; j0 += TNX) {
      T acc[4][MC];
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < MC; ++y) acc[x][y] = T(0);
      const bool active = (i0 + ti * 4 < M) && (j0 + tj * MC < N);
      // the next slab is read into registers while the current one is
      // multiplied from shared memory, so its global-memory latency is hidden
      constexpr int NA = kTK * kTM / kThreads, NB = kTK * TNX / kThreads;
      T ra[NA], rb[NB];
      auto load = [&](int k0) {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          const int e = tid + u * kThreads;
          int k, i;
          if (A_KFAST) { k = e % kTK; i = e / kTK; } else { i = e % kTM; k = e / kTM; }
          ra[u] = (i0 + i < M && k0 + k < K) ? T(fa(i0 + i, k0 + k)) : T(0);
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int e = tid + u * kThreads;
          int k, j;
          if (B_KFAST) { k = e % kTK; j = e / kTK; } else { j = e % TNX; k = e / TNX; }
          rb[u] = (j0 + j < N && k0 + k < K) ? T(fb(k0 + k, j0 + j)) : T(0);
        }
      };
      auto store = [&]() {
#pragma unroll
        for (int u = 0; u < NA; ++u) {
          const int e = tid + u * kThreads;
          int k, i;
          if (A_KFAST) { k = e % kTK; i = e / kTK; } else { i = e % kTM; k = e / kTM; }
          sA[k * kTM + i] = ra[u];
        }
#pragma unroll
        for (int u = 0; u < NB; ++u) {
          const int e = tid + u * kThreads;
          int k, j;
          if (B_KFAST) { k = e % kTK; j = e / kTK; } else { j = e % TNX; k = e / TNX; }
          sB[k * TNX + j] = rb[u];
        }
      };
      load(0);
      store();
      __syncthreads();
      for (int k0 = 0; k0 < K; k0 += kTK) {
        const bool more = k0 + kTK < K;
        if (more) load(k0 + kTK);
        if (active) {
          const int kk = min(kTK, K - k0);
          for (int k = 0; k < kk; ++k) {
            T a[4], bb[MC];
#pragma unroll
            for (int x = 0; x < 4; ++x) a[x] = sA[k * kTM + ti * 4 + x];
#pragma unroll
            for (int y = 0; y < MC; ++y) bb[y] = sB[k * TNX + tj * MC + y];
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < MC; ++y) acc[x][y] = fma(a[x], bb[y], acc[x][y]);
          }
        }
        __syncthreads();
        if (more) {
          store();
          __syncthreads();
        }
      }
      if (active) {
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < MC; ++y) {
            int i = i0 + ti * 4 + x, j = j0 + tj * MC + y;
            if (i < M && j < N) fc(i, j, double(acc[x][y]));
          }
      }
    }
  }
}

// Tc = tc::Split<NS>: the product runs on the tensor cores (tc_gemm.cuh)
// with NS BF16 slices per operand and FP32 accumulation.
template <class T> struct TcSlices { static constexpr int value = 0; };
template <int NS> struct TcSlices<tc::Split<NS>> { static constexpr int value = NS; };

// dynamic shared memory (doubles) of one product of arithmetic T
template <class T> __host__ __device__ constexpr int gemm_words() {
  return TcSlices<T>::value ? tc::smem_words<(TcSlices<T>::value ? TcSlices<T>::value : 1)>() : kGemmSmem;
}
template <class T> __host__ __device__ constexpr int tn_words();

// Dynamic shared memory of a product kernel: what its FP64 form needs, and at
// least the tensor-core product's stages for Tc = tc::Split.
template <class Tc> inline int tc_smem(int bytes) {
  return std::max(bytes, TcSlices<Tc>::value ? gemm_words<Tc>() * (int)sizeof(double) : 0);
}


// cta_gemm_t with the output tile width picked from N, or the tensor-core
// product for Tc = tc::Split<NS> (flags: the error word its bounded waits
// report to).
template <bool A_KFAST, bool B_KFAST, class T = double, class FA, class FB, class FC>
__device__ __forceinline__ void cta_gemm(int M, int N, int K, FA fa, FB fb, FC fc, double *smem,
                                         int *flags = nullptr) {
  constexpr int ns = TcSlices<T>::value;
  if constexpr (ns > 0) {
    tc::gemm<ns, A_KFAST, B_KFAST>(M, N, K, fa, fb, fc, smem, flags);
  } else {
    if (N <= 32) cta_gemm_t<T, A_KFAST, B_KFAST, 32>(M, N, K, fa, fb, fc, smem);
    else cta_gemm_t<T, A_KFAST, B_KFAST, 64>(M, N, K, fa, fb, fc, smem);
  }
}

// C(i, j) = sum_k A(k, i) B(k, j) for small outputs (M x N) and long K: the
// K rows are staged 32 at a time (coalesced along k), warp w takes rows
// w, w+4, ..., lanes own outputs (up to 16 each per pass), and the four
// warps' partial sums are added in a fixed order.  smem must hold
// 32 * (M + N) + 4 * 512 doubles; M + N <= kTnMaxMN.
constexpr int kTnMaxMN = 192;
constexpr int kTnSmem = 32 * kTnMaxMN + 4 * 512;
template <class T = double, class FA, class FB, class FC>
__device__ void cta_gemm_tn_simt(int M, int N, int K, FA fa, FB fb, FC fc, double *smem) {
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  T *sA = reinterpret_cast<T *>(smem);  // 32 x M  (sA[k * M + i])
  T *sB = sA + 32 * M;                  // 32 x N
  T *part = sB + 32 * N;                // 4 x 512 partial sums
  const int MN = M * N;
  for (int o0 = 0; o0 < MN; o0 += 512) {
    const int no = min(512, MN - o0);
    T acc[16];
#pragma unroll
    for (int u = 0; u < 16; ++u) acc[u] = T(0);
    for (int k0 = 0; k0 < K; k0 += 32) {
      const int kk = min(32, K - k0);
      for (int e = tid; e < 32 * M; e += kThreads) {
        int k = e & 31, i = e >> 5;
        sA[k * M + i] = (k < kk) ? T(fa(k0 + k, i)) : T(0);
      }
      for (int e = tid; e < 32 * N; e += kThreads) {
        int k = e & 31, j = e >> 5;
        sB[k * N + j] = (k < kk) ? T(fb(k0 + k, j)) : T(0);
      }
      __syncthreads();
      for (int k = warp; k < kk; k += 4) {
#pragma unroll
        for (int u = 0; u < 16; ++u) {
          int o = o0 + lane + 32 * u;
          if (o < o0 + no) {
            int i = o % M, j = o / M;
            acc[u] = fma(sA[k * M + i], sB[k * N + j], acc[u]);
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 16; ++u) part[warp * 512 + lane + 32 * u] = acc[u];
    __syncthreads();
    for (int e = tid; e < no; e += kThreads) {
      T v = ((part[e] + part[512 + e]) + part[1024 + e]) + part[1536 + e];
      int o = o0 + e;
      fc(o % M, o / M, double(v));
    }
    __syncthreads();
  }
}

template <class T> __host__ __device__ constexpr int tn_words() {
  return TcSlices<T>::value ? tc::smem_words<(TcSlices<T>::value ? TcSlices<T>::value : 1)>() : kTnSmem;
}

// C(i, j) = sum_k A(k, i) B(k, j), both operands contiguous along k: the
// small-output product above, or the tensor-core product for Tc = tc::Split.
template <class T = double, class FA, class FB, class FC>
__device__ __forceinline__ void cta_gemm_tn(int M, int N, int K, FA fa, FB fb, FC fc, double *smem,
                                            int *flags = nullptr) {
  constexpr int ns = TcSlices<T>::value;
  if constexpr (ns > 0) {
    tc::gemm<ns, true, true>(
        M, N, K, [&](int i, int k) { return fa(k, i); }, fb, fc, smem, flags);
  } else {
    cta_gemm_tn_simt<T>(M, N, K, fa, fb, fc, smem);
  }
}

// Sample width of the randomised compression of target block blk: the ACA
// rank of C_T plus the oversampling, capped at r.
__device__ __forceinline__ int sample_width(const FactorArgs &F, int blk) {
  int k = F.rank_c[blk];
  return min(F.r, max(8, k) + F.osamp);
}

// --- block accessors -----------------------------------------------------

struct Acc {
  const FactorArgs &F;
  __device__ Acc(const FactorArgs &f) : F(f) {}
  __device__ int kof(const BlockDesc &B) const { return B.kind == kLowRank ? F.kcap : F.b; }
  // columns of U_X that can be nonzero: the rank of a low-rank block of L, the
  // column count of a dense block
  __device__ int keff(int blk, const BlockDesc &B) const {
    return B.kind == kLowRank ? F.rank_l[blk] : B.cend - B.cbeg;
  }
  // U_X(row, col), row a global point index inside the block's rows
  __device__ double U(const BlockDesc &B, int row, int col) const {
    if (B.kind == kLowRank)
      return F.U[B.off_u + (row - B.rbeg) + (int64_t)col * (B.rend - B.rbeg)];
    return col < (B.cend - B.cbeg) ? F.D[B.off_d + (row - B.rbeg) + (int64_t)col * F.b] : 0.0;
  }
  // W_X(row, col), low-rank X, row a global point index inside the columns
  __device__ double W(const BlockDesc &B, int row, int col) const {
    const PanelDesc &P = F.panels[B.panel];
    return F.W[P.off + (row - P.rbeg) + (int64_t)(B.slot + col) * (P.rend - P.rbeg)];
  }
  __device__ double *Wp(int panel, int row, int col) const {
    const PanelDesc &P = F.panels[panel];
    return F.W + P.off + (row - P.rbeg) + (int64_t)col * (P.rend - P.rbeg);
  }
};

// --- P1 -------------------------------------------------------------------
// One CTA per row chunk of a gram G = W_A[ov]^T W_B[ov] (ranks x ranks).
template <class Tc>
__global__ void __launch_bounds__(kThreads) k_gram(FactorArgs Fz, int c0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  const GramChunk ch = F.gchunks[c0 + blockIdx.x];
  const GramTask g = F.grams[ch.g];
  const BlockDesc A = F.blocks[g.a], B = F.blocks[g.b];
  double *out = F.ws + ch.out;
  const int kc = F.kcap;
  const PanelDesc PA = F.panels[A.panel], PB = F.panels[B.panel];
  const int lda = PA.rend - PA.rbeg, ldb = PB.rend - PB.rbeg;
  const double *wa = F.W + PA.off + (int64_t)A.slot * lda + (ch.r0 - PA.rbeg);
  const double *wb = F.W + PB.off + (int64_t)B.slot * ldb + (ch.r0 - PB.rbeg);
  cta_gemm_tn<Tc>(
      F.rank_l[g.a], F.rank_l[g.b], ch.r1 - ch.r0, [&](int k, int i) { return wa[k + (int64_t)i * lda]; },
      [&](int k, int j) { return wb[k + (int64_t)j * ldb]; },
      [&](int i, int j, double v) { out[i + (int64_t)j * kc] = v; }, smem, F.flags);
}

// Sum of the chunks of a gram, in chunk order.
__global__ void __launch_bounds__(kThreads) k_gram_reduce(FactorArgs Fz, int r0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  const GramReduce R = F.greds[r0 + blockIdx.x];
  const GramTask g = F.grams[R.g];
  const int kc = F.kcap, ka = F.rank_l[g.a], kb = F.rank_l[g.b];
  for (int e = threadIdx.x; e < ka * kb; e += blockDim.x) {
    const int i = e % ka, j = e / ka;
    double v = 0.0;
    for (int c = 0; c < R.nchunk; ++c) v += F.ws[R.poff + (int64_t)c * kc * kc + i + j * kc];
    F.ws[g.goff + i + j * kc] = v;
  }
}

// --- P2a / P4a: t = U_X[rows]^T X[rows] for side entries; t_C for targets --
// trans = 0: B-entries against Omega (rows in sigma), t_C = V_C^T Omega.
// trans = 1: A-entries against Q (rows in rho), t_C = U_C^T Q.
template <class Tc>
__global__ void __launch_bounds__(kThreads) k_side_t(FactorArgs Fz, int e0, int ne, int t0, int trans) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  if ((int)blockIdx.x < ne) {
    const SideEntry E = trans ? F.aent[e0 + blockIdx.x] : F.bent[e0 + blockIdx.x];
    const LrTarget L = F.lrt[E.target];
    const int r = sample_width(F, L.blk);
    const BlockDesc T = F.blocks[L.blk];
    const BlockDesc X = F.blocks[E.blk];
    const int cb = trans ? T.rbeg : T.cbeg, ce = trans ? T.rend : T.cend;
    const int lo = max(cb, X.rbeg), hi = min(ce, X.rend);
    const int k = a.kof(X), ke = a.keff(E.blk, X);
    double *t = F.ws + E.toff;
    const double *Q = F.ws + L.yoff;
    const uint64_t seed = F.seed;
    const int64_t tb = L.blk;
    if (trans) {
      cta_gemm_tn<Tc>(
          ke, r, hi - lo, [&](int kk, int i) { return a.U(X, lo + kk, i); },
          [&](int kk, int j) { return Q[(lo + kk - cb) + (int64_t)j * L.m]; },
          [&](int i, int j, double v) { t[i + (int64_t)j * k] = v; }, smem, F.flags);
    } else {
      cta_gemm_tn<Tc>(
          ke, r, hi - lo, [&](int kk, int i) { return a.U(X, lo + kk, i); },
          [&](int kk, int j) { return rademacher(seed, tb, lo + kk - cb, j); },
          [&](int i, int j, double v) { t[i + (int64_t)j * k] = v; }, smem, F.flags);
    }
  } else {
    const LrTarget L = F.lrt[t0 + blockIdx.x - ne];
    const BlockDesc T = F.blocks[L.blk];
    const int r = sample_width(F, L.blk);
    const int kc = F.kc, kce = F.rank_c[L.blk];
    const double *UC = F.uc + (trans ? T.off_uc : T.off_vc);
    const int ld = trans ? L.m : L.p;
    double *tc = F.ws + L.tcoff;
    const double *Q = F.ws + L.yoff;
    const uint64_t seed = F.seed;
    const int64_t tb = L.blk;
    if (trans) {
      cta_gemm_tn<Tc>(
          kce, r, L.m, [&](int kk, int i) { return UC[kk + (int64_t)i * ld]; },
          [&](int kk, int j) { return Q[kk + (int64_t)j * L.m]; },
          [&](int i, int j, double v) { tc[i + (int64_t)j * kc] = v; }, smem, F.flags);
    } else {
      cta_gemm_tn<Tc>(
          kce, r, L.p, [&](int kk, int i) { return UC[kk + (int64_t)i * ld]; },
          [&](int kk, int j) { return rademacher(seed, tb, kk, j); },
          [&](int i, int j, double v) { tc[i + (int64_t)j * kc] = v; }, smem, F.flags);
    }
  }
}

// --- P2b / P4b: s_X = sum over the entry's pairs of L_q t_q ----------------
// Each pair q of the entry contributes a left factor L_q (rows of X x K_q)
// times the partner's t_q (K_q x r).  The pairs are concatenated along K (in
// chunks of at most kMaxRowK columns and kSidePairs pairs) into one product
// per CTA (the small-output, long-K product: rows of X x samples), in Tc
// arithmetic.
//   !trans (X = A, partner B)         trans (X = B, partner A)
//   LR/LR       L = G_AB                L = G_AB^T
//   A dense     L(i,k) = W_B(J0_A+i,k)   L(i,k) = W_B(J0_A+k,i)
//   B dense     L(i,k) = W_A(J0_B+k,i)   L(i,k) = W_A(J0_B+i,k)
//   both dense  L = I (the overlapping columns)
// Rows of a low-rank X beyond its rank are zero.
constexpr int kSidePairs = 256;
enum { kLG = 0, kLGt = 1, kLWik = 2, kLWki = 3, kLI = 4 };

template <class Tc>
__global__ void __launch_bounds__(kThreads) k_side_s(FactorArgs Fz, int e0, int trans) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  __shared__ int kb[kSidePairs + 1];
  __shared__ int pcase[kSidePairs], pnr[kSidePairs], pky[kSidePairs], pwld[kSidePairs];
  __shared__ int64_t pmat[kSidePairs], ptoff[kSidePairs];
  __shared__ short kmap[kMaxRowK];
  __shared__ int s_q1, s_nc;
  Acc a(F);
  const int kc = F.kcap;
  const SideEntry E = trans ? F.bent[e0 + blockIdx.x] : F.aent[e0 + blockIdx.x];
  const int r = sample_width(F, F.lrt[E.target].blk);
  const BlockDesc X = F.blocks[E.blk];
  const int kx = a.kof(X), kxe = a.keff(E.blk, X);
  const int M = X.kind == kDense ? kx : kxe;   // rows of s that can be nonzero
  double *s = F.ws + E.soff;
  const int32_t *plist = trans ? F.bpair : F.apair;
  for (int o = threadIdx.x; o < kx * r; o += blockDim.x)
    if (o % kx >= M || E.p1 == E.p0) s[o] = 0.0;
  int q0 = E.p0;
  bool first = true;
  while (q0 < E.p1) {
    if (threadIdx.x == 0) {   // describe the next chunk of pairs
      int k = 0, c = 0, q = q0;
      for (; q < E.p1 && c < kSidePairs; ++q) {
        const LrPair P = F.lrpairs[plist[q]];
        const int oe = trans ? P.ae : P.be;
        const SideEntry O = trans ? F.aent[oe] : F.bent[oe];
        const BlockDesc Y = F.blocks[O.blk];
        const BlockDesc &A = trans ? Y : X;
        const BlockDesc &B = trans ? X : Y;
        const int kye = a.keff(O.blk, Y);
        int cs, K, nr = 0, wld = 0;
        int64_t mat = 0;
        if (A.kind == kLowRank && B.kind == kLowRank) {
          cs = trans ? kLGt : kLG; K = kye; mat = P.goff;
        } else if (A.kind == kDense && B.kind == kDense) {
          cs = kLI; K = 0; nr = A.cend - A.cbeg;   // added directly after the product
        } else {
          const BlockDesc &Wb = (A.kind == kDense) ? B : A;   // the low-rank block holding W
          const PanelDesc PW = F.panels[Wb.panel];
          wld = PW.rend - PW.rbeg;
          const int J0 = (A.kind == kDense) ? A.cbeg : B.cbeg;
          const int nj = (A.kind == kDense) ? A.cend - A.cbeg : B.cend - B.cbeg;
          mat = PW.off + (int64_t)Wb.slot * wld + (J0 - PW.rbeg);   // W(J0 + x, y) = W[mat + x + y wld]
          const bool ik = (A.kind == kDense) != (trans != 0);      // L(i,k) = W(J0+i, k)?
          cs = ik ? kLWik : kLWki;
          K = ik ? kye : nj;
          nr = ik ? nj : 0;
        }
        if (k + K > kMaxRowK && c > 0) break;
        kb[c] = k; pcase[c] = cs; pnr[c] = nr; pmat[c] = mat; pwld[c] = wld;
        ptoff[c] = O.toff; pky[c] = a.kof(Y);
        k += K;
        ++c;
      }
      kb[c] = k;
      s_nc = c;
      s_q1 = q;
    }
    __syncthreads();
    const int nc = s_nc, K = min(kb[nc], kMaxRowK);
    for (int c = 0; c < nc; ++c)
      for (int k = kb[c] + threadIdx.x; k < min(kb[c + 1], K); k += blockDim.x) kmap[k] = (short)c;
    __syncthreads();
    const bool acc = !first;
    cta_gemm_tn<Tc>(
        M, r, K,
        [&](int k, int i) -> double {
          const int c = kmap[k], kk = k - kb[c];
          switch (pcase[c]) {
            case kLG: return F.ws[pmat[c] + i + (int64_t)kk * kc];
            case kLGt: return F.ws[pmat[c] + kk + (int64_t)i * kc];
            case kLWik: return i < pnr[c] ? F.W[pmat[c] + i + (int64_t)kk * pwld[c]] : 0.0;
            case kLWki: return F.W[pmat[c] + kk + (int64_t)i * pwld[c]];
            default: return 0.0;   // identity pairs take no columns
          }
        },
        [&](int k, int j) -> double {
          const int c = kmap[k];
          return F.ws[ptoff[c] + (k - kb[c]) + (int64_t)j * pky[c]];
        },
        [&](int i, int j, double v) {
          double *o = s + i + (int64_t)j * kx;
          *o = acc ? *o + v : v;
        },
        smem, F.flags);
    __syncthreads();
    // identity pairs (both blocks dense): s(i, j) += t_q(i, j), in pair order
    for (int o = threadIdx.x; o < M * r; o += blockDim.x) {
      const int i = o % M, j = o / M;
      double v = s[i + (int64_t)j * kx];
      for (int c = 0; c < nc; ++c)
        if (pcase[c] == kLI && i < pnr[c]) v += F.ws[ptoff[c] + i + (int64_t)j * pky[c]];
      s[i + (int64_t)j * kx] = v;
    }
    __syncthreads();
    q0 = s_q1;
    first = false;
  }
}

// --- P2c / P4c: rows of Y (or Z) of one leaf --------------------------------
template <class Tc>
__global__ void __launch_bounds__(kThreads) k_rows(FactorArgs Fz, int rt0, int trans) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  // per segment q of the concatenated K (q = 0: U_C, q >= 1: the entries):
  // the first column's left factor on the leaf's first row, its column
  // stride, the right factor's first row and its column stride
  __shared__ int kbeg[kMaxEntries + 2];
  __shared__ const double *ap[kMaxEntries + 2];
  __shared__ const double *bp[kMaxEntries + 2];
  __shared__ int ald[kMaxEntries + 2], bld[kMaxEntries + 2];
  __shared__ short kmap[kMaxRowK];          // column k of the concatenation -> segment
  Acc a(F);
  const int kc = F.kc;
  const RowTask R = trans ? F.brow[rt0 + blockIdx.x] : F.arow[rt0 + blockIdx.x];
  const LrTarget L = F.lrt[R.target];
  const int r = sample_width(F, L.blk);
  const BlockDesc T = F.blocks[L.blk];
  const int I0 = F.leaf_beg[R.leaf], I1 = F.leaf_beg[R.leaf + 1];
  const int base = trans ? T.cbeg : T.rbeg;
  const int ld = trans ? L.p : L.m;
  double *Y = F.ws + (trans ? L.zoff : L.yoff);
  const int mi = I1 - I0;
  const int32_t *ents = trans ? F.brow_ent : F.arow_ent;
  const int ne = R.e1 - R.e0;
  // K = [rank_c | k_e1 | k_e2 | ...]: Y[I] = [U_C[I], -U_e1[I], ...] [t_C; s_e1; ...]
  for (int q = threadIdx.x; q < ne; q += blockDim.x) {
    const SideEntry E = trans ? F.bent[ents[R.e0 + q]] : F.aent[ents[R.e0 + q]];
    const BlockDesc X = F.blocks[E.blk];
    if (X.kind == kLowRank) {
      ap[q + 1] = F.U + X.off_u + (I0 - X.rbeg);
      ald[q + 1] = X.rend - X.rbeg;
    } else {
      ap[q + 1] = F.D + X.off_d + (I0 - X.rbeg);
      ald[q + 1] = F.b;
    }
    bp[q + 1] = F.ws + E.soff;
    bld[q + 1] = a.kof(X);
    kbeg[q + 1] = a.keff(E.blk, X);   // segment lengths first, prefix sums below
  }
  if (threadIdx.x == 0) {
    ap[0] = F.uc + (trans ? T.off_vc : T.off_uc) + (I0 - base);
    ald[0] = ld;
    bp[0] = F.ws + L.tcoff;
    bld[0] = kc;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int k = F.rank_c[L.blk];
    kbeg[0] = 0;
    for (int q = 1; q <= ne; ++q) {
      const int len = kbeg[q];
      kbeg[q] = k;
      k += len;
    }
    kbeg[ne + 1] = k;
  }
  __syncthreads();
  const int K = min(kbeg[ne + 1], kMaxRowK);
  if (kbeg[ne + 1] > kMaxRowK && threadIdx.x == 0) raise_flag(F.flags, kFlagRankOverflow);
  for (int q = 0; q <= ne; ++q)
    for (int k = kbeg[q] + threadIdx.x; k < min(kbeg[q + 1], K); k += blockDim.x) kmap[k] = (short)q;
  __syncthreads();
  cta_gemm<false, true, Tc>(
      mi, r, K,
      [&](int i, int k) {
        const int q = kmap[k];
        const double v = ap[q][i + (int64_t)(k - kbeg[q]) * ald[q]];
        return q == 0 ? v : -v;
      },
      [&](int k, int j) {
        const int q = kmap[k];
        return bp[q][(k - kbeg[q]) + (int64_t)j * bld[q]];
      },
      [&](int i, int j, double v) { Y[(I0 - base + i) + (int64_t)j * ld] = v; }, smem, F.flags);
}

// --- tall QR (R factor only), then pivoted QR / SVD of the small R --------
constexpr int kQrRows = 64;

// R factor of the stacked h x r matrix A = [R; X] (ld h) in shared memory, in
// place: R (rows 0..r-1) is upper triangular with zeros below its diagonal,
// X holds rows r..h-1.  On return rows 0..r-1 hold the R factor of A; rows
// r..h-1 are overwritten.  Column j's reflector only involves row j and the
// rows of X (the rows of R below j are zero), so only those rows are read.
// The reflector is applied without being stored: w_c = A(j,c) + scal
// sum_i A(i,j) A(i,c), A(j,c) -= tau w_c, A(i,c) -= tau w_c scal A(i,j).
// Every warp computes the scalars of a column itself (lane 0, broadcast by
// shuffle), so a column costs one block reduction and one barrier.
__device__ void smem_householder(double *A, int h, int r, double *red) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int j = 0; j < r; ++j) {
    double s = 0.0;
    for (int i = r + threadIdx.x; i < h; i += blockDim.x) s = fma(A[i + j * h], A[i + j * h], s);
    s = block_sum(s, red);               // ends with a barrier: column j is final
    if (!(s > 0.0)) continue;            // nothing below the diagonal (uniform branch)
    double tau = 0.0, scal = 0.0, beta = 0.0;
    if (lane == 0) {                     // reflector scalars, once per warp
      const double alpha = A[j + j * h];
      const double nrm = sqrt(fma(alpha, alpha, s));
      beta = alpha >= 0.0 ? -nrm : nrm;
      tau = (beta - alpha) / beta;
      scal = 1.0 / (alpha - beta);
    }
    tau = __shfl_sync(0xffffffffu, tau, 0);
    scal = __shfl_sync(0xffffffffu, scal, 0);
    beta = __shfl_sync(0xffffffffu, beta, 0);
    for (int c = j + 1 + warp; c < r; c += nw) {
      double w = 0.0;
      for (int i = r + lane; i < h; i += 32) w = fma(A[i + j * h], A[i + c * h], w);
      w = warp_sum(w);
      w = tau * fma(scal, w, A[j + c * h]);
      if (lane == 0) A[j + c * h] -= w;
      const double ws = w * scal;
      for (int i = r + lane; i < h; i += 32) A[i + c * h] = fma(-ws, A[i + j * h], A[i + c * h]);
    }
    __syncthreads();                     // every column c > j is updated
    if (threadIdx.x == 0) A[j + j * h] = beta;
  }
  __syncthreads();
}

// R factor of one row group of a target's Y (which = 0) or Z (which = 1):
// rows are streamed 64 at a time below the running R, each block
// re-triangularised by Householder reflections.
__global__ void __launch_bounds__(kThreads) k_tsqr_part(FactorArgs Fz, int t0, int which) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  __shared__ double red[32];
  const LrTarget L = F.lrt[t0 + blockIdx.x];
  const int m = which ? L.p : L.m;
  const int G = which ? L.gp : L.gm;
  const int g = blockIdx.y;
  if (g >= G) return;
  const int r = sample_width(F, L.blk);
  const int h = r + kQrRows;
  const double *X = F.ws + (which ? L.zoff : L.yoff);
  const int len = (m + G - 1) / G;
  const int r0 = g * len, r1 = min(m, r0 + len);
  double *A = smem;  // h x r
  for (int e = threadIdx.x; e < h * r; e += blockDim.x) A[e] = 0.0;
  __syncthreads();
  for (int b0 = r0; b0 < r1; b0 += kQrRows) {
    const int rows = min(kQrRows, r1 - b0);
    for (int e = threadIdx.x; e < kQrRows * r; e += blockDim.x) {
      int i = e % kQrRows, c = e / kQrRows;
      A[(r + i) + c * h] = (i < rows) ? X[(b0 + i) + (int64_t)c * m] : 0.0;
    }
    // clear reflector data left below the diagonal of R
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      int i = e % r, c = e / r;
      if (i > c) A[i + c * h] = 0.0;
    }
    __syncthreads();
    smem_householder(A, h, r, red);
  }
  double *R = F.ws + L.roff + (int64_t)g * r * r;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int i = e % r, c = e / r;
    R[e] = (i <= c) ? A[i + c * h] : 0.0;
  }
}

// Column-pivoted Householder QR of the r x r matrix B (ld lb) in shared
// memory, in place: B P = Q R.  At step j the remaining column of largest
// norm is swapped in; the sweep stops where that norm falls below 1e-14 of
// the first pivot's (the rest is numerically zero).  On return rows 0..k1-1
// hold R in their upper triangle, piv the permutation (column j of B P is
// column piv[j] of B), and the result is k1.  Reflector scalars are computed
// once by thread 0; a column with nothing below its diagonal is left as it
// is (H = I).
struct PqrShared {
  int p, k1;
  double first, tau, beta;
};

__device__ int smem_pivoted_qr(double *B, int lb, int r, int *piv, double *cn, PqrShared &S) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  for (int c = threadIdx.x; c < r; c += blockDim.x) piv[c] = c;
  for (int c = warp; c < r; c += nw) {     // initial column norms, a warp per column
    double v = 0.0;
    for (int i = lane; i < r; i += 32) v = fma(B[i + c * lb], B[i + c * lb], v);
    v = warp_sum(v);
    if (lane == 0) cn[c] = v;
  }
  if (threadIdx.x == 0) { S.k1 = r; S.first = 0.0; }
  __syncthreads();
  for (int j = 0; j < r; ++j) {
    if (warp == 0) {   // pivot: largest remaining norm (ties -> lowest index)
      double bv = -1.0;
      int bi = j;
      for (int c = j + lane; c < r; c += 32)
        if (cn[c] > bv) { bv = cn[c]; bi = c; }
      for (int o = 16; o > 0; o >>= 1) {
        const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ov > bv || (ov == bv && oi < bi)) { bv = ov; bi = oi; }
      }
      if (lane == 0) {
        if (j == 0) S.first = bv;
        S.p = bi;
        if (!(bv > 1e-28 * S.first) || !(bv > 0.0)) S.k1 = j;   // the rest is rank deficient
      }
    }
    __syncthreads();
    if (S.k1 == j) break;
    const int p = S.p;
    if (p != j) {   // swap columns j and p (all rows), their norms and permutation entries
      for (int i = threadIdx.x; i < r; i += blockDim.x) {
        double t = B[i + j * lb]; B[i + j * lb] = B[i + p * lb]; B[i + p * lb] = t;
      }
      if (threadIdx.x == 0) {
        int t = piv[j]; piv[j] = piv[p]; piv[p] = t;
        double u = cn[j]; cn[j] = cn[p]; cn[p] = u;
      }
      __syncthreads();
    }
    if (warp == 0) {   // reflector for column j, rows j..r-1
      double s2 = 0.0;
      for (int i = j + 1 + lane; i < r; i += 32) s2 = fma(B[i + j * lb], B[i + j * lb], s2);
      s2 = warp_sum(s2);
      const double alpha = B[j + j * lb];
      double scal = 0.0;
      if (s2 > 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, s2));
        const double beta = alpha >= 0.0 ? -nrm : nrm;
        scal = 1.0 / (alpha - beta);
        if (lane == 0) { S.beta = beta; S.tau = (beta - alpha) / beta; }
      } else if (lane == 0) {   // nothing below the diagonal: H = I
        S.beta = alpha;
        S.tau = 0.0;
      }
      for (int i = j + 1 + lane; i < r; i += 32) B[i + j * lb] *= scal;
    }
    __syncthreads();
    const double tau = S.tau;
    // apply to the columns right of j, a warp per column; the same pass gives
    // each column's norm over rows j+1.. for the next pivot choice
    for (int c = j + 1 + warp; c < r; c += nw) {
      double w = 0.0;
      for (int i = j + 1 + lane; i < r; i += 32) w = fma(B[i + j * lb], B[i + c * lb], w);
      w = tau * (warp_sum(w) + B[j + c * lb]);
      double v2 = 0.0;
      for (int i = j + 1 + lane; i < r; i += 32) {
        const double x = fma(-w, B[i + j * lb], B[i + c * lb]);
        B[i + c * lb] = x;
        v2 = fma(x, x, v2);
      }
      v2 = warp_sum(v2);
      if (lane == 0) {
        B[j + c * lb] -= w;
        cn[c] = v2;
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) B[j + j * lb] = S.beta;
    __syncthreads();
  }
  return S.k1;
}

// Combine the row groups' R factors of Y (which = 0) or Z (which = 1) into
// one r x r R, then its column-pivoted QR R P = Q_r R_p with k1 kept pivots.
// mode 0 (orthonormalise): M = P_{:,1:k1} R_p11^{-1}, so that Q1 = Y M.
// mode 1 (truncate): the singular values and right singular vectors of R by
// one-sided Jacobi on R_p^T; k = smallest rank whose tail energy
// sum_{i>=k} sigma_i^2 is <= eps^2 max(sum sigma_i^2, |C_T|_F^2), or the
// leading fixed_k directions in the fixed-rank mode; M = V_k (r x kcap),
// k to rank_l.
__global__ void __launch_bounds__(kThreads) k_tsqr_final(FactorArgs Fz, int t0, int which, int mode) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  __shared__ double red[32];
  __shared__ int s_rot;
  __shared__ int ord[kMaxSample + 2];
  __shared__ double sig[kMaxSample + 2];
  __shared__ int s_rank;
  const LrTarget L = F.lrt[t0 + blockIdx.x];
  const int G = which ? L.gp : L.gm;
  const int r = sample_width(F, L.blk);
  const int ldm = F.r;                  // leading dimension of M in the workspace
  const int h = r + kQrRows;
  const int lb = r | 1;          // odd leading dimension: lane-per-column access is conflict free
  double *A = smem;              // h x r
  double *B = A + h * r;         // r x r (columns rotated), ld lb
  double *V = B + lb * r;        // r x r, ld lb
  for (int e = threadIdx.x; e < h * r; e += blockDim.x) A[e] = 0.0;
  __syncthreads();
  const int per = kQrRows / r > 0 ? kQrRows / r : 1;
  for (int g0 = 0; g0 < G; g0 += per) {
    const int cnt = min(per, G - g0);
    for (int e = threadIdx.x; e < kQrRows * r; e += blockDim.x) {
      int i = e % kQrRows, c = e / kQrRows;
      int gg = g0 + i / r, ii = i % r;
      A[(r + i) + c * h] = (i / r < cnt) ? F.ws[L.roff + (int64_t)gg * r * r + ii + c * r] : 0.0;
    }
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
      int i = e % r, c = e / r;
      if (i > c) A[i + c * h] = 0.0;
    }
    __syncthreads();
    smem_householder(A, h, r, red);
  }
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int i = e % r, c = e / r;
    B[i + c * lb] = (i <= c) ? A[i + c * h] : 0.0;
    V[i + c * lb] = (i == c) ? 1.0 : 0.0;
  }
  __syncthreads();
  __shared__ int piv[kMaxSample + 2];
  __shared__ double cn[kMaxSample + 2];
  __shared__ PqrShared pq;
  const int k1 = smem_pivoted_qr(B, lb, r, piv, cn, pq);
  if (mode == 0) {
    // Orthonormalisation: Q1 = Y P_{:,1:k1} R_p11^{-1} (the CholQR pass that
    // follows restores orthogonality to rounding level).
    // V <- R_p11^{-1} (upper triangular, k1 x k1), one thread per column
    for (int c = threadIdx.x; c < k1; c += blockDim.x) {
      for (int i = k1 - 1; i >= 0; --i) {
        double v = (i == c) ? 1.0 : 0.0;
        for (int l = i + 1; l <= c; ++l) v = fma(-B[i + l * lb], V[l + c * lb], v);
        V[i + c * lb] = (i <= c) ? v / B[i + i * lb] : 0.0;
      }
    }
    __syncthreads();
    double *M = F.ws + L.soff + ldm * ldm;
    for (int e = threadIdx.x; e < r * r; e += blockDim.x) M[(e % r) + (e / r) * ldm] = 0.0;
    __syncthreads();
    for (int e = threadIdx.x; e < k1 * k1; e += blockDim.x) {
      const int c = e / k1, q = e % k1;        // M(piv[q], c) = R_p11^{-1}(q, c)
      M[piv[q] + c * ldm] = V[q + c * lb];
    }
    if (threadIdx.x == 0) F.kept[t0 + blockIdx.x] = k1;
    return;
  }
  // mode 1: the SVD of R from the pivoted factor (R P = Q_r R_p): one-sided
  // Jacobi on the columns of X = R_p^T (its first k1 columns; the rest is
  // numerically zero).  The columns of X become U_X Sigma with R_p = V_X
  // Sigma U_X^T, so the right singular vectors of R are P U_X: no rotation
  // needs to be accumulated, and the pivoting leaves X's columns nearly
  // orthogonal, so few sweeps are needed.
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {   // X = R_p^T into V (scratch)
    const int c = e % r, i = e / r;                         // X(c, i) = R_p(i, c)
    V[c + i * lb] = (i < k1 && i <= c) ? B[i + c * lb] : 0.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) B[e % r + (e / r) * lb] = V[e % r + (e / r) * lb];
  __syncthreads();
  // A round rotates the disjoint column pairs of a round-robin tournament;
  // each pair is handled by a group of g lanes (all four warps busy, so all
  // four FP64 pipes of the SM), the group's lanes split the rows, and the
  // rotation parameters are computed once per group and broadcast.
  const int nc = k1;
  const int rp = nc + (nc & 1), half = rp / 2;
  double fro = 0.0;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    double v = B[e % r + (e / r) * lb];
    fro = fma(v, v, fro);
  }
  fro = block_sum(fro, red);
  const double tiny = 1e-30 * fro;     // columns below eps |R|_F are zero
  int g = 1;                            // lanes per pair: largest power of 2 with half * g <= 128
  while (g < 32 && half * g * 2 <= kThreads) g *= 2;
  const int grp = threadIdx.x / g, gl = threadIdx.x % g;
  double jf = 0.0;
  for (int sweep = 0; sweep < 40 && nc > 1; ++sweep) {
    __syncthreads();                    // every thread has read the previous flag
    if (threadIdx.x == 0) s_rot = 0;
    __syncthreads();
    for (int round = 0; round < rp - 1; ++round) {
      bool active = grp < half;
      int p = 0, q = 0;
      if (active) {
        p = (grp == 0) ? 0 : 1 + (grp - 1 + round) % (rp - 1);
        q = 1 + (rp - 2 - grp + round) % (rp - 1);
        if (p > q) { int t = p; p = q; q = t; }
        active = q < nc;
      }
      double al = 0.0, be = 0.0, ga = 0.0;
      if (active) {
        for (int i = gl; i < r; i += g) {
          double bp = B[i + p * lb], bq = B[i + q * lb];
          al = fma(bp, bp, al);
          be = fma(bq, bq, be);
          ga = fma(bp, bq, ga);
        }
      }
      for (int o = g / 2; o > 0; o >>= 1) {
        al += __shfl_xor_sync(0xffffffffu, al, o);
        be += __shfl_xor_sync(0xffffffffu, be, o);
        ga += __shfl_xor_sync(0xffffffffu, ga, o);
      }
      double c = 1.0, sn = 0.0;
      int rot = 0;
      if (active && gl == 0 && al > tiny && be > tiny && fabs(ga) > 1e-13 * sqrt(al * be)) {
        double zeta = (be - al) / (2.0 * ga);
        double t = (zeta >= 0.0 ? 1.0 : -1.0) / (fabs(zeta) + sqrt(fma(zeta, zeta, 1.0)));
        c = 1.0 / sqrt(fma(t, t, 1.0));
        sn = c * t;
        rot = 1;
        jf += 30.0;
      }
      const int src = (threadIdx.x & 31) / g * g;
      rot = __shfl_sync(0xffffffffu, rot, src);
      c = __shfl_sync(0xffffffffu, c, src);
      sn = __shfl_sync(0xffffffffu, sn, src);
      if (active && gl == 0) jf += 6.0 * r;
      if (active && rot) {
        for (int i = gl; i < r; i += g) {
          double bp = B[i + p * lb], bq = B[i + q * lb];
          B[i + p * lb] = c * bp - sn * bq;
          B[i + q * lb] = sn * bp + c * bq;
        }
        if (gl == 0) {
          s_rot = 1;
          jf += 6.0 * r;
        }
      }
      __syncthreads();
    }
    if (s_rot == 0) break;
  }
  jf = block_sum(jf, red);
  if (threadIdx.x == 0 && F.jacobi_flops) atomicAdd(F.jacobi_flops, jf);
  // V(piv[c], j) = X(c, j) / sigma_j: the right singular vectors of R
  for (int j = threadIdx.x; j < r; j += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < r; ++i) s = fma(B[i + j * lb], B[i + j * lb], s);
    sig[j] = sqrt(s);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    const int c = e % r, j = e / r;
    V[piv[c] + j * lb] = (sig[j] > 0.0) ? B[c + j * lb] / sig[j] : 0.0;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 0; i < r; ++i) ord[i] = i;
    for (int i = 0; i < r; ++i) {
      int best = i;
      for (int j = i + 1; j < r; ++j)
        if (sig[ord[j]] > sig[ord[best]]) best = j;
      int t = ord[i]; ord[i] = ord[best]; ord[best] = t;
    }
    {
      // truncate relative to the larger of |S| and |C_block|: C~ itself is
      // only accurate to eps |C_block| (ACA), so smaller singular values of
      // the updated block are noise
      double total = 0.0;
      for (int i = 0; i < r; ++i) total += sig[i] * sig[i];
      const double cnb = F.cnorm[L.blk];
      const double thr = F.eps * F.eps * fmax(total, cnb * cnb);
      int k = r;
      double tail = 0.0;
      while (k > 0) {
        double s2 = sig[ord[k - 1]] * sig[ord[k - 1]];
        if (tail + s2 > thr) break;
        tail += s2;
        --k;
      }
      if (!(total > 0.0)) k = 0;
      if (F.fixed_k > 0) {
        // fixed-rank mode (the rank-fixed approximation of Sec. 2): the
        // leading fixed_k directions whatever the accuracy, never an overflow
        k = 0;
        while (k < r && sig[ord[k]] > 1e-14 * sig[ord[0]]) ++k;
        k = min(k, min(F.fixed_k, F.kcap));
      } else {
        if (k > F.kcap) { raise_flag(F.flags, kFlagRankOverflow); k = F.kcap; }
        // too few samples left to trust the numerical rank
        if (k > r - F.osamp / 2) raise_flag(F.flags, kFlagRankOverflow);
      }
      s_rank = k;
      F.rank_l[L.blk] = k;
    }
  }
  __syncthreads();
  double *M = F.ws + L.soff + ldm * ldm;
  {
    const int k = s_rank, kc = F.kcap;
    for (int e = threadIdx.x; e < r * kc; e += blockDim.x) {
      int i = e % r, c = e / r;
      M[i + c * ldm] = (c < k) ? V[i + ord[c] * lb] : 0.0;
    }
  }
}

// Re-orthonormalisation of Q1 = Y P R_p11^{-1} (nearly orthonormal kept
// columns): partial Grams Q1_g^T Q1_g of the row groups ...
__global__ void __launch_bounds__(kThreads) k_cholqr_part(FactorArgs Fz, int t0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  const LrTarget L = F.lrt[t0 + blockIdx.x];
  const int G = L.gm, g = blockIdx.y;
  if (g >= G) return;
  const int r = sample_width(F, L.blk);
  const int k1 = F.kept[t0 + blockIdx.x];
  const int m = L.m, len = (m + G - 1) / G;
  const int r0 = g * len, r1 = min(m, r0 + len);
  const double *Q = F.ws + L.yoff;
  double *out = F.ws + L.roff + (int64_t)g * r * r;
  cta_gemm_tn(
      k1, k1, max(r1 - r0, 0), [&](int k, int i) { return Q[(r0 + k) + (int64_t)i * m]; },
      [&](int k, int j) { return Q[(r0 + k) + (int64_t)j * m]; },
      [&](int i, int j, double v) { out[i + j * r] = v; }, smem);
}

// ... then G = sum_g, G = R^T R (Cholesky), M = R^{-1} (k1 x k1, zero
// elsewhere) so that Q = Q1 M.
__global__ void __launch_bounds__(kThreads) k_cholqr_final(FactorArgs Fz, int t0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  __shared__ double s_inv;
  const LrTarget L = F.lrt[t0 + blockIdx.x];
  const int r = sample_width(F, L.blk), ldm = F.r;
  const int k1 = F.kept[t0 + blockIdx.x];
  double *Gs = smem;              // k1 x k1, ld r
  double *Ri = smem + r * r;      // R^{-1}, ld r
  for (int e = threadIdx.x; e < k1 * k1; e += blockDim.x) {
    int i = e % k1, j = e / k1;
    double v = 0.0;
    for (int g = 0; g < L.gm; ++g) v += F.ws[L.roff + (int64_t)g * r * r + i + j * r];
    Gs[i + j * r] = v;
  }
  __syncthreads();
  // Cholesky G = R^T R, R upper: column-oriented on the lower factor L = R^T
  for (int j = 0; j < k1; ++j) {
    if (threadIdx.x == 0) {
      double d = Gs[j + j * r];
      double l = sqrt(d > 0.0 ? d : 1.0);
      if (!(d > 0.0)) raise_flag(F.flags, kFlagNonFinite);
      Gs[j + j * r] = l;
      s_inv = 1.0 / l;
    }
    __syncthreads();
    for (int i = j + 1 + threadIdx.x; i < k1; i += blockDim.x) Gs[i + j * r] *= s_inv;
    __syncthreads();
    const int nt = k1 - j - 1;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
      int i = j + 1 + e % nt, l = j + 1 + e / nt;
      if (l <= i) Gs[i + l * r] = fma(-Gs[i + j * r], Gs[l + j * r], Gs[i + l * r]);
    }
    __syncthreads();
  }
  // inverse of the lower factor Lc (Lc Lc^T = G); R = Lc^T, so R^{-1} = (Lc^{-1})^T.
  // Column c of Lc^{-1} by forward substitution (one thread per column).
  for (int c = threadIdx.x; c < k1; c += blockDim.x) {
    for (int i = 0; i < k1; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int l = c; l < i; ++l) v = fma(-Gs[i + l * r], Ri[l + c * r], v);
      Ri[i + c * r] = (i < c) ? 0.0 : v / Gs[i + i * r];
    }
  }
  __syncthreads();
  double *M = F.ws + L.soff + ldm * ldm;
  for (int e = threadIdx.x; e < r * r; e += blockDim.x) {
    int i = e % r, j = e / r;     // M = (Lc^{-1})^T: M(i, j) = Ri(j, i)
    M[i + j * ldm] = (i < k1 && j < k1) ? Ri[j + i * r] : 0.0;
  }
}

// mode 0: Y <- Y M in place (r columns) for row chunk blockIdx.y.
// mode 1: U_T = Q V_k (rows of rho) and W_T = Z V_k (rows of sigma); the
//         chunk index runs over rho's chunks, then sigma's.
__global__ void __launch_bounds__(kThreads) k_tall_apply(FactorArgs Fz, int t0, int mode) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  const LrTarget L = F.lrt[t0 + blockIdx.x];
  const BlockDesc T = F.blocks[L.blk];
  const int r = sample_width(F, L.blk), ldm = F.r, kc = F.kcap;
  const double *M = F.ws + L.soff + ldm * ldm;
  const int chunk = blockIdx.y;
  if (mode == 0) {
    const int i0 = chunk * kTM;
    if (i0 >= L.m) return;
    const int mi = min(kTM, L.m - i0);
    double *Y = F.ws + L.yoff;
    cta_gemm<false, false>(
        mi, r, r, [&](int i, int k) { return Y[(i0 + i) + (int64_t)k * L.m]; },
        [&](int k, int j) { return M[k + j * ldm]; },
        [&](int i, int j, double v) { Y[(i0 + i) + (int64_t)j * L.m] = v; }, smem);
  } else {
    const int nch_m = (L.m + kTM - 1) / kTM;
    const int nch_p = (L.p + kTM - 1) / kTM;
    if (chunk < nch_m) {
      const int i0 = chunk * kTM, mi = min(kTM, L.m - i0);
      const double *Q = F.ws + L.yoff;
      double *U = F.U + T.off_u;
      cta_gemm<false, false>(
          mi, kc, r, [&](int i, int k) { return Q[(i0 + i) + (int64_t)k * L.m]; },
          [&](int k, int j) { return M[k + j * ldm]; },
          [&](int i, int j, double v) { U[(i0 + i) + (int64_t)j * L.m] = v; }, smem);
    } else if (chunk < nch_m + nch_p) {
      const int i0 = (chunk - nch_m) * kTM, mi = min(kTM, L.p - i0);
      const double *Z = F.ws + L.zoff;
      cta_gemm<false, false>(
          mi, kc, r, [&](int i, int k) { return Z[(i0 + i) + (int64_t)k * L.p]; },
          [&](int k, int j) { return M[k + j * ldm]; },
          [&](int i, int j, double v) { *a.Wp(T.panel, T.cbeg + i0 + i, T.slot + j) = v; },
          smem);
    }
  }
}

// --- P6: dense targets of column K -----------------------------------------
// k_dense_pair: one CTA per pair (A, B) of the step's dense targets writes
// P = U_A G_AB U_B^T restricted to the target (m x p, ld b) into the step's
// workspace; k_dense_reduce: S = C_IK - sum of the target's P in pair order.
template <class Tc>
__global__ void __launch_bounds__(kThreads) k_dense_pair(FactorArgs Fz, int q0, int64_t dpws) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  const int b = F.b, kc = F.kcap;
  const int q = q0 + blockIdx.x;
  const DPair Pq = F.dpairs[q];
  const BlockDesc A = F.blocks[Pq.a], B = F.blocks[Pq.b];
  double *out = F.ws + dpws + (int64_t)blockIdx.x * b * b;
  // the target's rows and columns (point ranges), stored per pair
  const int tr0 = F.dpair_tr[q].x, m = F.dpair_tr[q].y - F.dpair_tr[q].x;
  const int tc0 = F.dpair_tc[q].x, p = F.dpair_tc[q].y - F.dpair_tc[q].x;
  double *X = smem + gemm_words<Tc>();  // up to max(kcap, b) x b, ld ldx
  const int ldx = max(b, kc);
  auto put = [&](int i, int j, double v) { out[i + (int64_t)j * b] = v; };
  if (A.kind == kDense && B.kind == kDense) {
    const int nj = A.cend - A.cbeg;
    cta_gemm<false, true, Tc>(
        m, p, nj, [&](int i, int k) { return a.U(A, tr0 + i, k); },
        [&](int k, int j) { return a.U(B, tc0 + j, k); }, put, smem, F.flags);
    return;
  }
  int kx;
  if (A.kind == kLowRank && B.kind == kLowRank) {
    kx = F.rank_l[Pq.a];
    const int kb = F.rank_l[Pq.b];
    const double *G = F.ws + Pq.goff;
    cta_gemm<false, true, Tc>(
        kx, p, kb, [&](int i, int k) { return G[i + (int64_t)k * kc]; },
        [&](int k, int j) { return a.U(B, tc0 + j, k); },
        [&](int i, int j, double v) { X[i + j * ldx] = v; }, smem, F.flags);
  } else if (A.kind == kDense) {  // B low-rank: X = W_B[J_A] U_B[K]^T
    kx = A.cend - A.cbeg;
    const int J0 = A.cbeg;
    cta_gemm<false, true, Tc>(
        kx, p, F.rank_l[Pq.b], [&](int i, int k) { return a.W(B, J0 + i, k); },
        [&](int k, int j) { return a.U(B, tc0 + j, k); },
        [&](int i, int j, double v) { X[i + j * ldx] = v; }, smem, F.flags);
  } else {  // A low-rank, B dense: X = W_A[J_B]^T D_B^T
    kx = F.rank_l[Pq.a];
    const int J0 = B.cbeg, nj = B.cend - B.cbeg;
    cta_gemm<true, true, Tc>(
        kx, p, nj, [&](int i, int k) { return a.W(A, J0 + k, i); },
        [&](int k, int j) { return a.U(B, tc0 + j, k); },
        [&](int i, int j, double v) { X[i + j * ldx] = v; }, smem, F.flags);
  }
  __syncthreads();
  const int kxx = kx;
  cta_gemm<false, false, Tc>(
      m, p, kxx, [&](int i, int k) { return a.U(A, tr0 + i, k); },
      [&](int k, int j) { return X[k + j * ldx]; }, put, smem, F.flags);
}

__global__ void __launch_bounds__(kThreads) k_dense_reduce(FactorArgs Fz, int d0, int64_t dpws) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  const int b = F.b;
  const DenseTarget DT = F.dns[d0 + blockIdx.x];
  const BlockDesc T = F.blocks[DT.blk];
  const int m = T.rend - T.rbeg, p = T.cend - T.cbeg;
  const int q0 = F.dns[d0].p0;
  double *S = F.D + T.off_d;
  const double *Cb = F.Cd + T.off_d;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e % b, j = e / b;
    double v = 0.0;
    if (i < m && j < p) {
      v = Cb[e];
      for (int q = DT.p0; q < DT.p1; ++q) v -= F.ws[dpws + (int64_t)(q - q0) * b * b + e];
    }
    S[e] = v;
  }
}

// --- P7: Cholesky of the diagonal leaf ------------------------------------
__global__ void __launch_bounds__(kThreads) k_potrf(FactorArgs Fz, int d0, int K) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  const int b = F.b;
  const DenseTarget DT = F.dns[d0];
  const BlockDesc T = F.blocks[DT.blk];
  const int m = T.rend - T.rbeg;
  double *G = F.D + T.off_d;
  double *A = smem;  // m x m, ld b
  __shared__ double red[32];
  __shared__ int bad;
  __shared__ double s_inv;
  if (threadIdx.x == 0) bad = 0;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) A[e] = G[e];
  __syncthreads();
  for (int j = 0; j < m; ++j) {
    if (threadIdx.x == 0) {
      double djj = A[j + j * b];
      if (!(djj > 0.0) || !isfinite(djj)) { bad = 1; djj = 1.0; }
      double l = sqrt(djj);
      A[j + j * b] = l;
      s_inv = 1.0 / l;
    }
    __syncthreads();
    const double inv = s_inv;
    for (int i = j + 1 + threadIdx.x; i < m; i += blockDim.x) A[i + j * b] *= inv;
    __syncthreads();
    const int nt = m - j - 1;
    for (int e = threadIdx.x; e < nt * nt; e += blockDim.x) {
      int i = j + 1 + e % nt, l = j + 1 + e / nt;
      if (l <= i) A[i + l * b] = fma(-A[i + j * b], A[l + j * b], A[i + l * b]);
    }
    __syncthreads();
  }
  double s = 0.0;
  for (int j = threadIdx.x; j < m; j += blockDim.x) s += log(A[j + j * b]);
  s = block_sum(s, red);
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) {
    int i = e % b, l = e / b;
    G[e] = (i >= l && i < m) ? A[e] : 0.0;
  }
  if (threadIdx.x == 0) {
    F.logdet_parts[K] = 2.0 * s;
    if (bad) raise_flag(F.flags, kFlagNotSpd);
  }
}

// --- P8: off-diagonal dense blocks of column K: X = S L^{-T} ---------------
__global__ void __launch_bounds__(kThreads) k_trsm(FactorArgs Fz, int d0, int K) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  const int b = F.b;
  const BlockDesc Dg = F.blocks[F.dns[d0].blk];
  const int mk = Dg.rend - Dg.rbeg;
  double *Lk = smem;  // b x b
  double *rdiag = smem + b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) Lk[e] = F.D[Dg.off_d + e];
  for (int j = threadIdx.x; j < mk; j += blockDim.x) rdiag[j] = 1.0 / F.D[Dg.off_d + j + j * b];
  __syncthreads();
  const DenseTarget DT = F.dns[d0 + 1 + blockIdx.x];
  const BlockDesc T = F.blocks[DT.blk];
  const int m = T.rend - T.rbeg;
  double *S = F.D + T.off_d;
  for (int i = threadIdx.x; i < m; i += blockDim.x) {
    for (int j = 0; j < mk; ++j) {
      double v = S[i + j * b];
      for (int l = 0; l < j; ++l) v = fma(-S[i + l * b], Lk[j + l * b], v);
      S[i + j * b] = v * rdiag[j];
    }
  }
}

// --- P9: W <- L_KK^{-1} W on the rows of leaf K of each open panel --------
__global__ void __launch_bounds__(kThreads) k_wsolve(FactorArgs Fz, int w0, int d0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  const int b = F.b;
  const BlockDesc Dg = F.blocks[F.dns[d0].blk];
  const int mk = Dg.rend - Dg.rbeg;
  double *Lk = smem;
  double *rdiag = smem + b * b;
  for (int e = threadIdx.x; e < b * b; e += blockDim.x) Lk[e] = F.D[Dg.off_d + e];
  for (int j = threadIdx.x; j < mk; j += blockDim.x) rdiag[j] = 1.0 / F.D[Dg.off_d + j + j * b];
  __syncthreads();
  const int pn = F.wpan[w0 + blockIdx.x];
  const PanelDesc P = F.panels[pn];
  const int ld = P.rend - P.rbeg;
  const int c0 = blockIdx.y * blockDim.x;
  const int c = c0 + threadIdx.x;
  if (c >= P.width) return;
  double *w = F.W + P.off + (Dg.rbeg - P.rbeg) + (int64_t)c * ld;
  double x[kMaxLeaf];
  for (int i = 0; i < mk; ++i) {
    double v = w[i];
    for (int l = 0; l < i; ++l) v = fma(-Lk[i + l * b], x[l], v);
    x[i] = v * rdiag[i];
  }
  for (int i = 0; i < mk; ++i) w[i] = x[i];
}

// --- P10a: H = W_A^T W_panel[cols A] -----------------------------------------
template <class Tc>
__global__ void __launch_bounds__(kThreads) k_htask(FactorArgs Fz, int h0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  const HTask H = F.hts[h0 + blockIdx.x];
  const BlockDesc A = F.blocks[H.a];
  const PanelDesc P = F.panels[H.panel];
  const int ld = P.rend - P.rbeg, kc = F.kcap;
  double *out = F.ws + H.hoff;
  const double *Wp = F.W + P.off;
  const int ka = F.rank_l[H.a];
  const PanelDesc PA = F.panels[A.panel];
  const int lda = PA.rend - PA.rbeg;
  const double *wa = F.W + PA.off + (int64_t)A.slot * lda + (A.cbeg - PA.rbeg);
  // column chunk blockIdx.y of the panel (chunks run in parallel CTAs)
  for (int j0 = blockIdx.y * (kTnMaxMN - kMaxRank); j0 < P.width; j0 += gridDim.y * (kTnMaxMN - kMaxRank)) {
    const int nj = min(kTnMaxMN - kMaxRank, P.width - j0);
    cta_gemm_tn<Tc>(
        ka, nj, A.cend - A.cbeg, [&](int k, int i) { return wa[k + (int64_t)i * lda]; },
        [&](int k, int j) { return Wp[(A.cbeg + k - P.rbeg) + (int64_t)(j0 + j) * ld]; },
        [&](int i, int j, double v) { out[i + (int64_t)(j0 + j) * kc] = v; }, smem, F.flags);
  }
}

// --- P10b: W_panel[I] -= sum of the leaf row's updates ----------------------
template <class Tc>
__global__ void __launch_bounds__(kThreads) k_updrow(FactorArgs Fz, int u0) {
  const FactorArgs F = Fz.at(blockIdx.z);   // evaluation blockIdx.z of the batch
  extern __shared__ double smem[];
  Acc a(F);
  const UpdRow R = F.urows[u0 + blockIdx.x];
  const PanelDesc P = F.panels[R.panel];
  const int ld = P.rend - P.rbeg, kc = F.kcap;
  const int I0 = F.leaf_beg[R.leaf], I1 = F.leaf_beg[R.leaf + 1];
  const int mi = I1 - I0;
  double *Wp = F.W + P.off;
  for (int q = R.e0; q < R.e1; ++q) {
    const UpdEntry E = F.uents[q];
    const BlockDesc A = F.blocks[E.a];
    __syncthreads();
    auto sub = [&](int i, int j, double v) { Wp[(I0 - P.rbeg + i) + (int64_t)j * ld] -= v; };
    if (E.hoff < 0) {
      const int nj = A.cend - A.cbeg;
      cta_gemm<false, false, Tc>(
          mi, P.width, nj, [&](int i, int k) { return a.U(A, I0 + i, k); },
          [&](int k, int j) { return Wp[(A.cbeg + k - P.rbeg) + (int64_t)j * ld]; }, sub, smem, F.flags);
    } else {
      const double *Hm = F.ws + E.hoff;
      cta_gemm<false, true, Tc>(
          mi, P.width, F.rank_l[E.a], [&](int i, int k) { return a.U(A, I0 + i, k); },
          [&](int k, int j) { return Hm[k + (int64_t)j * kc]; }, sub, smem, F.flags);
    }
  }
}

__global__ void k_permute_in(const double *__restrict__ z, const int32_t *__restrict__ perm,
                             int64_t n, double *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = z[perm[i]];
}

__global__ void k_finalize(const double *__restrict__ parts, int N, const double *__restrict__ w,
                           int64_t n, double *__restrict__ out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < N; i += blockDim.x) s += parts[i];
  s = block_sum(s, red);
  double q = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) q = fma(w[i], w[i], q);
  q = block_sum(q, red);
  if (threadIdx.x == 0) { out[0] = s; out[1] = q; }
}

int g_smem_bytes = 0;
int g_smem_dense = 0;

}  // namespace

__global__ void k_bw_h(FactorArgs F, const int32_t *blks, const double *__restrict__ v,
                       double *__restrict__ h);
__global__ void k_lmv_t(FactorArgs F, const int32_t *lr_ids, const double *__restrict__ x,
                        double *__restrict__ t);

int factor_smem_setup(int b, int kcap) {
  g_smem_bytes = (kGemmSmem + b * b) * (int)sizeof(double);
  int kx = b > kcap ? b : kcap;
  g_smem_dense = (kGemmSmem + kx * b) * (int)sizeof(double);
  cudaError_t e = cudaSuccess;
#define SETA(k, s) e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, s); if (e != cudaSuccess) return (int)e
  const int tn = kTnSmem * (int)sizeof(double);
#define SETA_TC(kern, bytes)                      \
  SETA(kern<double>, bytes);                      \
  SETA(kern<tc::Split<3>>, tc_smem<tc::Split<3>>(bytes)); \
  SETA(kern<tc::Split<2>>, tc_smem<tc::Split<2>>(bytes))
  SETA_TC(k_gram, g_smem_bytes);
  SETA_TC(k_side_t, g_smem_bytes);
  SETA_TC(k_side_s, tn);
  SETA_TC(k_rows, g_smem_bytes);
  SETA(k_tsqr_part, (kMaxSample + kQrRows) * kMaxSample * (int)sizeof(double));
  SETA(k_cholqr_part, kTnSmem * (int)sizeof(double));
  SETA(k_cholqr_final, 2 * kMaxSample * kMaxSample * (int)sizeof(double));
  SETA(k_tsqr_final, ((kMaxSample + kQrRows) * kMaxSample + 2 * (kMaxSample + 1) * kMaxSample) * (int)sizeof(double));
  SETA(k_tall_apply, g_smem_bytes);
  SETA(k_dense_pair<double>, g_smem_dense);
  SETA(k_dense_pair<tc::Split<3>>, (gemm_words<tc::Split<3>>() + kx * b) * (int)sizeof(double));
  SETA(k_dense_pair<tc::Split<2>>, (gemm_words<tc::Split<2>>() + kx * b) * (int)sizeof(double));
  SETA(k_potrf, g_smem_bytes);
  SETA(k_trsm, g_smem_bytes);
  SETA(k_wsolve, g_smem_bytes);
  SETA_TC(k_htask, g_smem_bytes);
  SETA_TC(k_updrow, g_smem_bytes);
#undef SETA_TC
  SETA(k_bw_h, kTnSmem * (int)sizeof(double));
  SETA(k_lmv_t, kTnSmem * (int)sizeof(double));
#undef SETA
  return 0;
}

const char *const kKernelNames[KK_COUNT] = {
    "k_gram", "k_side_t", "k_side_s", "k_rows", "k_tsqr_part", "k_tsqr_final", "k_tall_apply",
    "k_cholqr_part", "k_cholqr_final", "k_dense_pair", "k_dense_reduce", "k_potrf", "k_trsm",
    "k_wsolve", "k_htask", "k_updrow"};

void prof_mark(Prof *p, cudaStream_t s) {
  if ((int)p->ev.size() <= p->used) {
    cudaEvent_t e;
    cudaEventCreate(&e);
    p->ev.push_back(e);
  }
  cudaEventRecord(p->ev[p->used++], s);
}

void prof_collect(Prof *p, int nev) {
  for (int i = 0; i + 1 < nev; i += 2) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, p->ev[i], p->ev[i + 1]) == cudaSuccess) {
      p->ms += ms;
      ++p->launches;
    } else {
      const cudaError_t e = cudaGetLastError();  // do not leave it for an unrelated status check
      if (!p->failed++) p->first_err = (int)e;
    }
  }
}

#define LAUNCH(KIND, strm, ...)                                   \
  do {                                                            \
    const bool prof_on__ = prof && prof->kind == (KIND);          \
    if (prof_on__) prof_mark(prof, strm);                         \
    __VA_ARGS__;                                                  \
    if (prof_on__) prof_mark(prof, strm);                         \
    ++nk;                                                         \
  } while (0)

namespace {
// One step of the sweep.  Tl: arithmetic of the products of the low-rank
// targets' compression and of the deferred panel updates (k_side_t/s, k_rows,
// k_htask, k_updrow); Td: that of the Grams and of the dense targets' products
// (k_gram, k_dense_pair), the updates of the diagonal leaves.
template <class Tl, class Td>
int launch_step_t(cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join,
                  const FactorArgs &F, const StepRange &S, int K, const Plan &PL, Prof *prof) {
  const std::vector<LrTarget> &lrt_host = PL.lrt;
  int nk = 0;
  const int sm = (kGemmSmem + F.b * F.b) * (int)sizeof(double);
  const int smt = std::max(kGemmSmem + F.b * F.b, kTnSmem) * (int)sizeof(double);
  const int smd = (gemm_words<Td>() + std::max(F.b, F.kcap) * F.b) * (int)sizeof(double);
  const int stn = kTnSmem * (int)sizeof(double);    // a small-output product and nothing else
  const int r = F.r;
  if (S.gch1 > S.gch0) { LAUNCH(KK_GRAM, st, k_gram<Td><<<dim3(S.gch1 - S.gch0, 1, F.nz), kThreads, tc_smem<Td>(smt), st>>>(F, S.gch0)); }
  if (S.gred1 > S.gred0) { LAUNCH(KK_GRAM, st, k_gram_reduce<<<dim3(S.gred1 - S.gred0, 1, F.nz), kThreads, 0, st>>>(F, S.gred0)); }
  // the dense blocks of column K (P6-P8) only need the grams: fork them to
  // the side stream while the low-rank targets are compressed
  cudaStream_t sd = side ? side : st;
  if (side) {
    cudaEventRecord(ev_fork, st);
    cudaStreamWaitEvent(side, ev_fork, 0);
  }
  const int nd = S.dns1 - S.dns0;
  const int q0 = PL.dns[S.dns0].p0, q1 = PL.dns[S.dns1 - 1].p1;
  if (q1 > q0) { LAUNCH(KK_DENSE_PAIR, sd, k_dense_pair<Td><<<dim3(q1 - q0, 1, F.nz), kThreads, smd, sd>>>(F, q0, S.dpws)); }
  LAUNCH(KK_DENSE_REDUCE, sd, k_dense_reduce<<<dim3(nd, 1, F.nz), kThreads, 0, sd>>>(F, S.dns0, S.dpws));
  LAUNCH(KK_POTRF, sd, k_potrf<<<dim3(1, 1, F.nz), kThreads, sm, sd>>>(F, S.dns0, K));
  if (nd > 1) { LAUNCH(KK_TRSM, sd, k_trsm<<<dim3(nd - 1, 1, F.nz), kThreads, sm, sd>>>(F, S.dns0, K)); }
  const int nt = S.lrt1 - S.lrt0;
  if (nt > 0) {
    int maxch = 0, maxgm = 1, maxgp = 1;
    for (int t = S.lrt0; t < S.lrt1; ++t) {
      const LrTarget &L = lrt_host[t];
      int ch = (L.m + kTM - 1) / kTM + (L.p + kTM - 1) / kTM;
      if (ch > maxch) maxch = ch;
      maxgm = std::max(maxgm, L.gm);
      maxgp = std::max(maxgp, L.gp);
    }
    const int qr_smem = (r + kQrRows) * r * (int)sizeof(double);
    const int qrf_smem = ((r + kQrRows) * r + 2 * (r | 1) * r) * (int)sizeof(double);
    const int cq_smem = 2 * r * r * (int)sizeof(double);
    // Y = S Omega
    LAUNCH(KK_SIDE_T, st, k_side_t<Tl><<<dim3((S.bent1 - S.bent0) + nt, 1, F.nz), kThreads, tc_smem<Tl>(smt), st>>>(F, S.bent0, S.bent1 - S.bent0, S.lrt0, 0));
    if (S.aent1 > S.aent0) LAUNCH(KK_SIDE_S, st, k_side_s<Tl><<<dim3(S.aent1 - S.aent0, 1, F.nz), kThreads, tc_smem<Tl>(stn), st>>>(F, S.aent0, 0));
    LAUNCH(KK_ROWS, st, k_rows<Tl><<<dim3(S.arow1 - S.arow0, 1, F.nz), kThreads, tc_smem<Tl>(sm), st>>>(F, S.arow0, 0));
    // Q = orth(Y): R of Y, pivoted QR, Q1 = Y P R_p11^{-1}, then CholQR
    LAUNCH(KK_TSQR_PART, st, k_tsqr_part<<<dim3(nt, maxgm, F.nz), kThreads, qr_smem, st>>>(F, S.lrt0, 0));
    LAUNCH(KK_TSQR_FINAL, st, k_tsqr_final<<<dim3(nt, 1, F.nz), kThreads, qrf_smem, st>>>(F, S.lrt0, 0, 0));
    LAUNCH(KK_TALL_APPLY, st, k_tall_apply<<<dim3(nt, maxch, F.nz), kThreads, sm, st>>>(F, S.lrt0, 0));
    LAUNCH(KK_CHOLQR_PART, st, k_cholqr_part<<<dim3(nt, maxgm, F.nz), kThreads, kTnSmem * (int)sizeof(double), st>>>(F, S.lrt0));
    LAUNCH(KK_CHOLQR_FINAL, st, k_cholqr_final<<<dim3(nt, 1, F.nz), kThreads, cq_smem, st>>>(F, S.lrt0));
    LAUNCH(KK_TALL_APPLY, st, k_tall_apply<<<dim3(nt, maxch, F.nz), kThreads, sm, st>>>(F, S.lrt0, 0));
    // Z = S^T Q
    LAUNCH(KK_SIDE_T, st, k_side_t<Tl><<<dim3((S.aent1 - S.aent0) + nt, 1, F.nz), kThreads, tc_smem<Tl>(smt), st>>>(F, S.aent0, S.aent1 - S.aent0, S.lrt0, 1));
    if (S.bent1 > S.bent0) LAUNCH(KK_SIDE_S, st, k_side_s<Tl><<<dim3(S.bent1 - S.bent0, 1, F.nz), kThreads, tc_smem<Tl>(stn), st>>>(F, S.bent0, 1));
    LAUNCH(KK_ROWS, st, k_rows<Tl><<<dim3(S.brow1 - S.brow0, 1, F.nz), kThreads, tc_smem<Tl>(sm), st>>>(F, S.brow0, 1));
    LAUNCH(KK_TSQR_PART, st, k_tsqr_part<<<dim3(nt, maxgp, F.nz), kThreads, qr_smem, st>>>(F, S.lrt0, 1));
    LAUNCH(KK_TSQR_FINAL, st, k_tsqr_final<<<dim3(nt, 1, F.nz), kThreads, qrf_smem, st>>>(F, S.lrt0, 1, 1));
    LAUNCH(KK_TALL_APPLY, st, k_tall_apply<<<dim3(nt, maxch, F.nz), kThreads, sm, st>>>(F, S.lrt0, 1));
  }
  if (side) {
    cudaEventRecord(ev_join, side);
    cudaStreamWaitEvent(st, ev_join, 0);
  }
  if (S.wpan1 > S.wpan0) {
    int maxw = 0;
    for (int q = S.wpan0; q < S.wpan1; ++q) maxw = std::max(maxw, PL.panels[PL.wpan[q]].width);
    LAUNCH(KK_WSOLVE, st, k_wsolve<<<dim3(S.wpan1 - S.wpan0, (maxw + kThreads - 1) / kThreads, F.nz), kThreads, sm, st>>>(
        F, S.wpan0, S.dns0));
  }
  if (S.ht1 > S.ht0) {
    int maxw = 1;
    for (int q = S.ht0; q < S.ht1; ++q) maxw = std::max(maxw, PL.panels[PL.hts[q].panel].width);
    const int ny = (maxw + (kTnMaxMN - kMaxRank) - 1) / (kTnMaxMN - kMaxRank);
    LAUNCH(KK_HTASK, st, k_htask<Tl><<<dim3(S.ht1 - S.ht0, ny, F.nz), kThreads, tc_smem<Tl>(smt), st>>>(F, S.ht0));
  }
  if (S.ur1 > S.ur0) { LAUNCH(KK_UPDROW, st, k_updrow<Tl><<<dim3(S.ur1 - S.ur0, 1, F.nz), kThreads, tc_smem<Tl>(sm), st>>>(F, S.ur0)); }
  return nk;
}
}  // namespace

int launch_step(cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join,
                const FactorArgs &F, const StepRange &S, int K, const Plan &PL, Prof *prof) {
  // the mixed forms run every product on the tensor cores: FP32-class
  // operands (three BF16 slices) or 16-bit operands (two slices)
  if (F.mixed == 1) return launch_step_t<tc::Split<3>, tc::Split<3>>(st, side, ev_fork, ev_join, F, S, K, PL, prof);
  if (F.mixed == 2) return launch_step_t<tc::Split<2>, tc::Split<2>>(st, side, ev_fork, ev_join, F, S, K, PL, prof);
  return launch_step_t<double, double>(st, side, ev_fork, ev_join, F, S, K, PL, prof);
}

// --- a17: y = L x (field simulation Z = L xi) ------------------------------
// t_A = W_A^T x[cols A] for every low-rank block of L ...
__global__ void __launch_bounds__(kThreads) k_lmv_t(FactorArgs F, const int32_t *lr_ids,
                                                     const double *__restrict__ x,
                                                     double *__restrict__ t) {
  extern __shared__ double smem[];
  Acc a(F);
  const int blk = lr_ids[blockIdx.x];
  const BlockDesc A = F.blocks[blk];
  cta_gemm_tn(
      F.rank_l[blk], 1, A.cend - A.cbeg, [&](int k, int i) { return a.W(A, A.cbeg + k, i); },
      [&](int k, int j) { return x[A.cbeg + k]; },
      [&](int i, int j, double v) { t[(int64_t)blk * F.kcap + i] = v; }, smem);
}

// ... then each leaf row sums its blocks: dense D x[cols] (the diagonal block
// is lower triangular) and U_A[I] t_A, in a fixed order.
__global__ void __launch_bounds__(kThreads) k_lmv_rows(FactorArgs F, const int32_t *row0,
                                                        const int32_t *rblocks,
                                                        const double *__restrict__ x,
                                                        const double *__restrict__ t,
                                                        double *__restrict__ y) {
  Acc a(F);
  const int I = blockIdx.x;
  const int I0 = F.leaf_beg[I], I1 = F.leaf_beg[I + 1];
  for (int i = I0 + threadIdx.x; i < I1; i += blockDim.x) {
    double acc = 0.0;
    for (int q = row0[I]; q < row0[I + 1]; ++q) {
      const int blk = rblocks[q];
      const BlockDesc B = F.blocks[blk];
      if (B.kind == kDense) {
        for (int j = 0; j < B.cend - B.cbeg; ++j) acc = fma(a.U(B, i, j), x[B.cbeg + j], acc);
      } else {
        for (int k = 0; k < F.rank_l[blk]; ++k) acc = fma(a.U(B, i, k), t[(int64_t)blk * F.kcap + k], acc);
      }
    }
    y[i] = acc;
  }
}

__global__ void k_permute_out(const double *__restrict__ y, const int32_t *__restrict__ perm,
                              int64_t n, double *__restrict__ out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[perm[i]] = y[i];
}

void launch_lower_matvec(cudaStream_t st, const FactorArgs &F, const int32_t *lr_ids, int nlr,
                         const int32_t *row0, const int32_t *rblocks, int nleaf,
                         const double *x, double *y, double *t) {
  const int smt = kTnSmem * (int)sizeof(double);
  if (nlr > 0) k_lmv_t<<<nlr, kThreads, smt, st>>>(F, lr_ids, x, t);
  k_lmv_rows<<<nleaf, kThreads, 0, st>>>(F, row0, rblocks, x, t, y);
}

void launch_solve(cudaStream_t st, const FactorArgs &F0, const Plan &PL, const int32_t *wpan_rhs) {
  FactorArgs F = F0;
  F.wpan = wpan_rhs;
  const int sm = (kGemmSmem + F.b * F.b) * (int)sizeof(double);
  const int smt = std::max(kGemmSmem + F.b * F.b, kTnSmem) * (int)sizeof(double);
  for (int K = 0; K < PL.nleaf; ++K) {
    const StepRange &S = PL.steps[K];
    k_wsolve<<<dim3(1, 1), kThreads, sm, st>>>(F, 0, S.dns0);
    const int h0 = PL.ht_rhs0[K], h1 = PL.ht_rhs0[K + 1];
    if (h1 > h0) k_htask<double><<<h1 - h0, kThreads, smt, st>>>(F, h0);
    const int u0 = PL.ur_rhs0[K], u1 = PL.ur_rhs0[K + 1];
    if (u1 > u0) k_updrow<double><<<u1 - u0, kThreads, sm, st>>>(F, u0);
  }
}

// --- a11: backward solve v = L^{-T} w --------------------------------------
// L^T is block upper triangular, so the leaves are solved in reverse order:
// v_K = L_KK^{-T} (w_K - sum over blocks A below the diagonal block of leaf K
// of A^T v[rows A]).  Once v_K is final, every block whose rows start at
// leaf K has all its rows final and pushes A^T v[rows A] into its columns.

// v_K <- L_KK^{-T} v_K by back substitution (one thread; m <= 128)
__global__ void k_bw_diag(FactorArgs F, int dblk, double *__restrict__ v) {
  const BlockDesc D = F.blocks[dblk];
  const int m = D.rend - D.rbeg, b = F.b;
  const double *L = F.D + D.off_d;   // column-major, leading dimension b
  if (threadIdx.x == 0) {
    for (int i = m - 1; i >= 0; --i) {
      double s = v[D.rbeg + i];
      for (int l = i + 1; l < m; ++l) s = fma(-L[l + (int64_t)i * b], v[D.rbeg + l], s);
      v[D.rbeg + i] = s / L[i + (int64_t)i * b];
    }
  }
}

// h_A = U_A^T v[rows A] for the low-rank blocks whose rows start at this leaf
__global__ void __launch_bounds__(kThreads) k_bw_h(FactorArgs F, const int32_t *blks,
                                                   const double *__restrict__ v,
                                                   double *__restrict__ h) {
  extern __shared__ double smem[];
  Acc a(F);
  const int blk = blks[blockIdx.x];
  const BlockDesc A = F.blocks[blk];
  cta_gemm_tn(
      F.rank_l[blk], 1, A.rend - A.rbeg, [&](int k, int i) { return a.U(A, A.rbeg + k, i); },
      [&](int k, int j) { return v[A.rbeg + k]; },
      [&](int i, int j, double val) { h[(int64_t)blockIdx.x * F.kcap + i] = val; }, smem);
}

// v[J] -= sum over the entries of column leaf J, in a fixed order: W_A[J] h_A
// for a low-rank block, D_A^T v[rows A] for a dense one.
__global__ void __launch_bounds__(kThreads) k_bw_upd(FactorArgs F, const UpdRow *rows,
                                                     const UpdEntry *ents,
                                                     const double *__restrict__ h,
                                                     double *__restrict__ v) {
  Acc a(F);
  const UpdRow R = rows[blockIdx.x];
  const int J0 = F.leaf_beg[R.leaf], J1 = F.leaf_beg[R.leaf + 1];
  for (int j = J0 + threadIdx.x; j < J1; j += blockDim.x) {
    double acc = 0.0;
    for (int q = R.e0; q < R.e1; ++q) {
      const UpdEntry E = ents[q];
      const BlockDesc A = F.blocks[E.a];
      if (E.hoff < 0) {
        for (int i = 0; i < A.rend - A.rbeg; ++i)
          acc = fma(a.U(A, A.rbeg + i, j - A.cbeg), v[A.rbeg + i], acc);
      } else {
        const double *hA = h + E.hoff * F.kcap;
        for (int k = 0; k < F.rank_l[E.a]; ++k) acc = fma(a.W(A, j, k), hA[k], acc);
      }
    }
    v[j] -= acc;
  }
}

void launch_backward(cudaStream_t st, const FactorArgs &F, const Plan &PL, double *v,
                     const int32_t *bh_blocks, const UpdRow *bupd, const UpdEntry *bents,
                     double *hbuf) {
  const int smt = kTnSmem * (int)sizeof(double);
  for (int K = PL.nleaf - 1; K >= 0; --K) {
    k_bw_diag<<<1, 32, 0, st>>>(F, PL.diag_of_leaf[K], v);
    const int h0 = PL.bh0[K], h1 = PL.bh0[K + 1];
    if (h1 > h0) k_bw_h<<<h1 - h0, kThreads, smt, st>>>(F, bh_blocks + h0, v, hbuf);
    const int u0 = PL.bupd0[K], u1 = PL.bupd0[K + 1];
    if (u1 > u0) k_bw_upd<<<u1 - u0, kThreads, 0, st>>>(F, bupd + u0, bents, hbuf, v);
  }
}

void launch_permute_out(cudaStream_t st, const double *y, const int32_t *perm, int64_t n,
                        double *out) {
  k_permute_out<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(y, perm, n, out);
}

void launch_permute_in(cudaStream_t st, const double *z, const int32_t *perm, int64_t n,
                       double *out) {
  k_permute_in<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(z, perm, n, out);
}

void launch_finalize(cudaStream_t st, const double *parts, int N, const double *w, int64_t n,
                     double *out) {
  k_finalize<<<1, 1024, 0, st>>>(parts, N, w, n, out);
}

}  // namespace hmle
