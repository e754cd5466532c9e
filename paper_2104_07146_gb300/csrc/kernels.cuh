// Kernel argument structs and launchers of libhmle (assemble.cu, factor.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "hmle_internal.h"

namespace hmle {

// θ-dependent scalars, kept in device memory so that a captured graph of
// the sweep stays valid across evaluations.
struct ThetaDev {
  double inv_ell, sigma2, tau2, nu;
};

struct AsmArgs {
  const BlockDesc *blocks;
  const int32_t *lr_ids;   // admissible block ids
  const double *xyz;       // cluster-order coordinates (SoA)
  int64_t n;
  int d;
  const double *tab;       // Matern table
  double inv_ell, sigma2, tau2, eps;
  int kc;
  double *uc;              // ACA pool (U and V of C)
  int32_t *rank_c;
  double *cnorm;           // |C_block|_F estimate of every admissible block
  int *flags;
  int fixed_k;             // > 0: fixed-rank mode, every block at most this rank
  const ThetaDev *thd;     // the same theta in device memory (read by captured kernels)
  const double *Cd;        // dense near-field blocks (b x b at each dense block's off_d)
  int b;                   // leaf size (leading dimension of the Cd blocks)
  // a batch: evaluation z's H-matrix buffers are evaluation 0's shifted by
  // z * zstride bytes (the H-matrix operator of the batched PCG)
  int64_t zstride;
  __host__ __device__ AsmArgs at(int z) const {
    AsmArgs G = *this;
    if (z == 0) return G;
    const int64_t o = (int64_t)z * zstride;
    auto sh = [o](auto *p) { return p ? reinterpret_cast<decltype(p)>(const_cast<char *>(reinterpret_cast<const char *>(p)) + o) : p; };
    G.tab = sh(tab); G.uc = sh(uc); G.rank_c = sh(rank_c); G.cnorm = sh(cnorm); G.flags = sh(flags);
    G.thd = sh(thd); G.Cd = sh(Cd);
    return G;
  }
};

// Everything the sweep kernels read; device pointers.
struct FactorArgs {
  const BlockDesc *blocks;
  const PanelDesc *panels;
  const GramTask *grams;
  const GramChunk *gchunks;
  const GramReduce *greds;
  const LrTarget *lrt;
  const SideEntry *aent, *bent;
  const int32_t *apair, *bpair;
  const LrPair *lrpairs;
  const RowTask *arow, *brow;
  const int32_t *arow_ent, *brow_ent;
  const DenseTarget *dns;
  const DPair *dpairs;
  const int2 *dpair_tr, *dpair_tc;  // target rows / columns of each dense pair
  const int32_t *wpan;
  const HTask *hts;
  const UpdRow *urows;
  const UpdEntry *uents;
  const int32_t *leaf_beg;  // first point of leaf K (N + 1 entries)
  // pools
  double *D;               // dense blocks of L (b x b each, ld b)
  const double *uc;        // ACA factors of C
  const double *Cd;        // dense near-field blocks of C (b x b at each dense block's off_d)
  const int32_t *rank_c;
  const double *cnorm;     // |C_block|_F of the admissible blocks (ACA)
  double *U;               // U factors of L
  double *W;               // W-panels (incl. the right-hand side)
  double *ws;              // per-step workspace
  int32_t *rank_l;
  int32_t *kept;           // per low-rank target: columns kept by the orthonormalisation
  double *jacobi_flops;    // FP64 flops of the Jacobi sweeps (data-dependent count)
  double *logdet_parts;    // per leaf
  int *flags;
  // geometry / kernel
  const double *xyz;
  int64_t n;
  int d;
  const double *tab;
  const ThetaDev *th;
  double eps;
  uint64_t seed;
  int b, kcap, kc, r;
  int osamp;               // oversampling of the randomised compression
  int fixed_k;             // > 0: fixed-rank mode (truncate at this rank, no overflow)
  int mixed;               // 0 FP64; 1, 2: the mixed forms (products on the tensor cores)
  // A batch of nz evaluations of one tree (different theta): every buffer of
  // evaluation z (the H-matrix of C, the factor, the workspace, the flags) is
  // that of evaluation 0 shifted by z * zstride bytes, and a sweep kernel
  // launched with gridDim.z = nz serves evaluation blockIdx.z.
  int nz;
  int64_t zstride;
  __host__ __device__ FactorArgs at(int z) const {
    FactorArgs G = *this;
    if (z == 0) return G;
    const int64_t o = (int64_t)z * zstride;
    G.D = shift(D, o); G.uc = shift(uc, o); G.Cd = shift(Cd, o); G.rank_c = shift(rank_c, o);
    G.cnorm = shift(cnorm, o); G.U = shift(U, o); G.W = shift(W, o); G.ws = shift(ws, o);
    G.rank_l = shift(rank_l, o); G.kept = shift(kept, o); G.jacobi_flops = shift(jacobi_flops, o);
    G.logdet_parts = shift(logdet_parts, o); G.flags = shift(flags, o); G.tab = shift(tab, o);
    G.th = shift(th, o);
    return G;
  }
  template <class P>
  __host__ __device__ static P *shift(P *p, int64_t o) {
    return p ? reinterpret_cast<P *>(const_cast<char *>(reinterpret_cast<const char *>(p)) + o) : p;
  }
};

void launch_matern_table(cudaStream_t st, double nu, double *tab);
void launch_matern_eval(cudaStream_t st, const double *tab, const double *x, int64_t m,
                        double *out);
void launch_aca(cudaStream_t st, const AsmArgs &A, int n_lr);
// dense near-field blocks of C into Cd (the dense blocks' b x b slots, off_d)
void launch_assemble_dense(cudaStream_t st, const AsmArgs &A, const int32_t *dense_ids, int nd,
                           int b, double *Cd);
// Kernel kinds of the sweep (for per-kernel timing and flop tallies).
enum KernelKind {
  KK_GRAM = 0, KK_SIDE_T, KK_SIDE_S, KK_ROWS, KK_TSQR_PART, KK_TSQR_FINAL, KK_TALL_APPLY,
  KK_CHOLQR_PART, KK_CHOLQR_FINAL, KK_DENSE_PAIR, KK_DENSE_REDUCE, KK_POTRF, KK_TRSM,
  KK_WSOLVE, KK_HTASK, KK_UPDROW, KK_COUNT
};
extern const char *const kKernelNames[KK_COUNT];

// Optional CUDA-event timing of one kernel kind: an event is recorded on the
// launching stream before and after every launch of that kind.
struct Prof {
  int kind = -1;
  std::vector<cudaEvent_t> ev;
  int used = 0;                 // events recorded by the current launch sequence
  double ms = 0.0;
  int64_t launches = 0;
  double flops = 0.0;
  int failed = 0;               // event pairs whose elapsed time could not be read
  int first_err = 0;            // the cudaError_t of the first such pair
};
void prof_mark(Prof *p, cudaStream_t s);
// after a stream synchronisation: add the elapsed times of the first nev
// events (pairs) and keep the pool for reuse
void prof_collect(Prof *p, int nev);

// One step K of the sweep (all phases), given the step's ranges.
// Returns the number of kernels launched.
// side / ev_fork / ev_join: a second stream (or nullptr) and two events used
// to run the dense blocks of the step concurrently with the low-rank targets.
int launch_step(cudaStream_t st, cudaStream_t side, cudaEvent_t ev_fork, cudaEvent_t ev_join,
                const FactorArgs &F, const StepRange &S, int K, const Plan &PL, Prof *prof);

void launch_permute_in(cudaStream_t st, const double *z, const int32_t *perm, int64_t n,
                       double *out);
// y = L x in cluster order (x, y: n doubles); t: workspace of kcap doubles
// per block; lr_ids / nlr: the low-rank blocks; row0 / rblocks: per leaf row
// the blocks covering it (device copies of Plan::mv_row0 / mv_blocks).
void launch_lower_matvec(cudaStream_t st, const FactorArgs &F, const int32_t *lr_ids, int nlr,
                         const int32_t *row0, const int32_t *rblocks, int nleaf,
                         const double *x, double *y, double *t);
// Forward solve w <- L^{-1} w on the right-hand-side panel of a finished
// factor (F's task pointers set to the rhs-only lists: hts/urows/uents;
// wpan must hold the rhs panel index at position 0).
void launch_solve(cudaStream_t st, const FactorArgs &F, const Plan &PL, const int32_t *wpan_rhs);
// Backward solve v <- L^{-T} v in place on a vector v (cluster order), by the
// reverse leaf sweep; hbuf: workspace of kcap doubles per low-rank block of
// the largest step.  bh_blocks / bupd / bents: device copies of the plan's
// backward lists.
void launch_backward(cudaStream_t st, const FactorArgs &F, const Plan &PL, double *v,
                     const int32_t *bh_blocks, const UpdRow *bupd, const UpdEntry *bents,
                     double *hbuf);
// out[perm[k]] = y[k]
void launch_permute_out(cudaStream_t st, const double *y, const int32_t *perm, int64_t n,
                        double *out);
// logdet = sum(parts[0..N)), quad = |w|^2; out[0] = logdet, out[1] = quad
void launch_finalize(cudaStream_t st, const double *parts, int N, const double *w, int64_t n,
                     double *out);
int factor_smem_setup(int b, int kcap);

// Fixed-order lists of the symmetric H-matvec y = C x (device pointers):
// per leaf I, the blocks whose rows cover I (row0 / rblocks, diagonal block
// first) and the off-diagonal blocks whose columns cover I (col0 / cblocks);
// lr_slot[blk] = index of blk among the admissible blocks, -1 if dense.
struct CmvLists {
  int nleaf;
  const int32_t *leaf_beg, *row0, *rblocks, *col0, *cblocks, *lr_slot;
};
// y = C x in cluster order (FP64; dense entries generated from the table);
// t: 2 kc doubles per admissible block.  A batch of nz: vectors x, y at
// z zs doubles, t at z tzs (tzs < 0: zs), the H-matrix A.at(z) (one
// H-matrix for all when A.zstride = 0).
void launch_cmatvec(cudaStream_t st, const AsmArgs &A, int n_lr, const CmvLists &L,
                    const double *x, double *t, double *y, int nz = 1, int64_t zs = 0, int64_t tzs = -1);
// Eq. 5-6 helpers.  Columns j0 .. j0 + cnt - 1 of C12 (no nugget):
// out[i + jj ld] = sigma2 M_nu(|s1_i - s2_{j0+jj}| inv_ell), i < n in cluster
// order (xyz SoA), locs2 m x d row-major.
void launch_cross_cols(cudaStream_t st, const double *tab, const double *xyz, int64_t n, int d,
                       const double *locs2, int64_t j0, int cnt, double inv_ell, double sigma2, double *out,
                       int64_t ld);
// out[jj] = sum_i a[i + jj ld] b[i + jj ld], i < n, for jj < cnt: one CTA per
// column, fixed order.
void launch_col_dots(cudaStream_t st, const double *a, const double *b, int64_t n, int64_t ld, int cnt,
                     double *out);
// doubles of workspace pcg_quad needs
int64_t pcg_words(int64_t n, int n_lr, int kc, int hmax);
// q = b^T x with C x = b solved by PCG: operator launch_cmatvec, preconditioner
// the factor of Fs (F's task pointers set to the right-hand-side lists) applied
// through the right-hand-side panel `panel` (overwritten).  b: n doubles,
// cluster order.  Stops when |r| <= tol |b| or after maxit iterations.
// Device copies of the per-leaf task lists of the two sweeps on one vector.
struct SolvePlan {
  int nleaf;
  const int32_t *diag;                    // diagonal block of each leaf
  const int32_t *ht0, *ur0;               // forward: per leaf ranges (nleaf + 1)
  const HTask *hts;                       // forward: right-hand-side panel tasks
  const UpdRow *urows;
  const UpdEntry *uents;
  const int32_t *bh0, *bu0;               // backward: per leaf ranges (nleaf + 1)
  const int32_t *bblk;                    // backward: low-rank blocks per leaf
  const UpdRow *bupd;
  const UpdEntry *bents;
};
// w <- L~^{-1} w (backward = false; h = the factor's workspace) or
// w <- L~^{-T} w (backward = true; h = kcap doubles per low-rank block of the
// largest leaf list) in one cooperative launch; bar: 3 unsigned of device
// memory for the grid barrier, bar[2] zeroed by the caller beforehand
// (bar[2] != 0 afterwards: a barrier wait ran out).
cudaError_t persistent_solve(cudaStream_t st, const FactorArgs &F, const SolvePlan &P, double *w,
                             double *h, unsigned *bar, bool backward);
// The same sweep for nrhs vectors of one factor in one cooperative launch:
// vector z at w + z ws, its coupling vectors at h + z hs.  P's forward task
// lists must address the coupling vectors compactly (the hmle_tree's
// multi-vector plan: kcap doubles per task of a leaf, hs >= the largest
// leaf's tasks x kcap in either direction).
cudaError_t persistent_solve_multi(cudaStream_t st, const FactorArgs &F, const SolvePlan &P, double *w,
                                   int64_t ws, double *h, int64_t hs, int nrhs, unsigned *bar, bool backward);

// Eq. 4: out[j] = sum_i sigma2 M_nu(|s2_j - s1_i| inv_ell) x_i for m new
// locations locs2 (m x d, row-major) against the n training points xyz (SoA,
// cluster order); x in cluster order.
void launch_cross_matvec(cudaStream_t st, const double *tab, const double *xyz, int64_t n, int d,
                         const double *locs2, int64_t m, double inv_ell, double sigma2,
                         const double *x, double *out);
// out[i] = sum_j sigma2 M_nu(|s1_i - s2_j| inv_ell) y_j (the transposed product;
// out in cluster order).
void launch_cross_matvec_t(cudaStream_t st, const double *tab, const double *xyz, int64_t n, int d,
                           const double *locs2, int64_t m, double inv_ell, double sigma2,
                           const double *y, double *out);

// One PCG solve C x = b (b: n doubles, cluster order) with q = b^T x:
// operator launch_cmatvec, preconditioner the factor of Fs (task pointers set
// to the right-hand-side lists) applied through the right-hand-side panel
// `panel` (overwritten); stops when |r| <= tol |b| or after maxit
// iterations.  The set-up and one iteration are captured as CUDA graphs into
// *g_init / *g_iter on first use when those are not NULL (the pointers and
// theta they read are fixed per buffer set; theta is read from device
// memory) and replayed afterwards.  host: 3 doubles of pinned memory for the
// scalars read back.  pcg_start launches the set-up and the first iteration;
// after each synchronisation of st, pcg_poll reads the residual and launches
// the next iteration or the final dot (then *finished once q is in).  Several
// solves on different streams can so run interleaved.
struct PcgRun {
  cudaStream_t st;
  const SolvePlan *SP;      // when not NULL: preconditioner by the persistent sweeps
  unsigned *bar;            // their barrier words (3 unsigned, device)
  AsmArgs A;
  int n_lr;
  CmvLists L;
  FactorArgs Fs;
  const Plan *PL;
  const int32_t *wpan_rhs, *bh_blocks;
  const UpdRow *bupd;
  const UpdEntry *bents;
  double *panel;
  const double *b;
  int64_t n;
  double tol;
  int maxit;
  double *pool;
  double *host;
  cudaGraphExec_t *g_init, *g_iter;
  // results
  int it = 0, state = 0;
  double rel = 1.0, q = 0.0;
  bool timed_out = false;   // a barrier wait of the persistent sweeps ran out
  // a batch of nz solves in lockstep (pcg_batch_*): evaluation z's vectors,
  // pool, panel and factor are evaluation 0's shifted by z zs doubles; each
  // stops updating its solution once it has converged (or reached maxit), as
  // a single solve would stop, and the batch runs until all have
  int nz = 1;
  int64_t zs = 0;
  double *hostz = nullptr;  // pinned: per evaluation 4 doubles (stopped, iterations, rel, q)
  std::vector<int> itz;     // per evaluation results of a batch
  std::vector<double> relz, qz;
};
cudaError_t pcg_batch_start(PcgRun &R);
cudaError_t pcg_batch_poll(PcgRun &R, bool *finished);
cudaError_t pcg_start(PcgRun &R);
cudaError_t pcg_poll(PcgRun &R, bool *finished);
cudaError_t pcg_quad(PcgRun &R);   // start, then synchronise and poll until finished

}  // namespace hmle
