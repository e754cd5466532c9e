// The C ABI of libhmle (include/hmle.h): handles, device memory,
// orchestration of the kernels, and the Nelder-Mead driver of hmle_fit.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <string>
#include <vector>

#include "common.cuh"
#include "hmle_internal.h"
#include "kernels.cuh"
#include "matern.cuh"
#include "tally.h"
#include "tree.cuh"

using namespace hmle;

struct hmle_ctx {
  cudaStream_t st = nullptr;
  bool own = false;
  int dev = 0;
  std::string err;
  cudaStream_t side = nullptr;     // dense blocks of a step run here concurrently
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  Prof prof;                       // optional per-kernel timing
  double *d_jacobi = nullptr;      // device flop counter of the Jacobi sweeps
};

struct DevPlan {
  BlockDesc *blocks = nullptr;
  PanelDesc *panels = nullptr;
  GramTask *grams = nullptr;
  GramChunk *gchunks = nullptr;
  GramReduce *greds = nullptr;
  LrTarget *lrt = nullptr;
  SideEntry *aent = nullptr, *bent = nullptr;
  int32_t *apair = nullptr, *bpair = nullptr;
  LrPair *lrpairs = nullptr;
  RowTask *arow = nullptr, *brow = nullptr;
  int32_t *arow_ent = nullptr, *brow_ent = nullptr;
  DenseTarget *dns = nullptr;
  DPair *dpairs = nullptr;
  int2 *dpair_tr = nullptr, *dpair_tc = nullptr;
  int32_t *wpan = nullptr;
  HTask *hts = nullptr;
  UpdRow *urows = nullptr;
  UpdEntry *uents = nullptr;
  int32_t *leaf_beg = nullptr;
  int32_t *lr_ids = nullptr;
  int32_t *dense_ids = nullptr;
  int32_t *mv_row0 = nullptr, *mv_blocks = nullptr;
  HTask *hts_rhs = nullptr;
  UpdRow *urows_rhs = nullptr;
  UpdEntry *uents_rhs = nullptr;
  int32_t *wpan_rhs = nullptr;
  int32_t *bh_blocks = nullptr;
  UpdRow *bupd = nullptr;
  UpdEntry *bents = nullptr;
  int32_t *mvt_row0 = nullptr, *mvt_blocks = nullptr, *lr_slot = nullptr;
  int32_t *diag = nullptr, *ht_rhs0 = nullptr, *ur_rhs0 = nullptr, *bh0 = nullptr, *bupd0 = nullptr;
  HTask *hts_mrhs = nullptr;       // the forward lists of the multi-vector sweep: coupling
  UpdEntry *uents_mrhs = nullptr;  // vectors at kcap doubles per task of the leaf
  int64_t bytes = 0;
};

struct Work;   // per-tree evaluation buffers (θ-dependent contents)
struct Group;  // a batch of evaluations of one tree whose buffers share one layout

struct hmle_tree {
  hmle_ctx *ctx = nullptr;   // used by calls on the tree; never by its destructor
  int64_t n = 0;
  int d = 2;
  hmle_opts opts{};
  Plan plan;
  DeviceTree T;
  DevPlan dp;
  std::vector<int32_t> lr_ids, dense_ids;
  Work *work = nullptr;
  std::vector<Work *> pool;  // evaluation buffers of hmle_loglik_multi
  std::vector<Group *> groups;  // the batch of hmle_loglik_batch (at most one, of the last size used)
  bool graphs = true;        // replay the sweep as a captured CUDA graph
  SolvePlan sp{};            // device task lists of the persistent sweeps on one vector
  SolvePlan spm{};           // the same for many vectors (compact coupling vectors)
  int64_t mrhs_h = 0;        // coupling-vector doubles per vector of the multi-vector sweeps
  bool coop = false;         // the device supports cooperative launches
  bool owns_T = true;        // false: T belongs to the tree this one was derived from
  std::vector<int4> blocks0; // block tree (level, i, j, kind) as built, for derived plans
  std::vector<int32_t> cb, ce;   // heap-indexed cluster ranges
};

struct hmle_hmatrix {
  const hmle_tree *tree = nullptr;
  hmle_theta th{};
  double *tab = nullptr;
  double *uc = nullptr;
  double *Cd = nullptr;       // dense near-field blocks of C (b x b at each dense block's off_d)
  int32_t *rank_c = nullptr;
  double *cnorm = nullptr;
  ThetaDev *thd = nullptr;
  int *flags = nullptr;
  int max_rank_c = 0;
  bool owned = true;
};

struct hmle_hfactor {
  const hmle_hmatrix *h = nullptr;
  double *D = nullptr, *U = nullptr, *W = nullptr, *ws = nullptr;
  int32_t *rank_l = nullptr;
  int32_t *kept = nullptr;
  double *ldp = nullptr;
  int *flags = nullptr;
  double *out = nullptr;
  bool has_rhs = false;
  double logdet = 0.0, quad = 0.0;
  double host_out[2] = {0.0, 0.0};   // results of an asynchronous evaluation
  int host_flags[2] = {0, 0};
  int64_t launches = 0;
  int max_rank_l = 0;
  double mean_rank_l = 0.0;
  bool owned = true;
  double *pcg = nullptr;      // mixed form: right-hand side + PCG workspace
  double *pcg_host = nullptr; // pinned scalars read back by the PCG
  cudaGraphExec_t pcg_init = nullptr, pcg_iter = nullptr;   // its captured sequences
  int pcg_iters = 0;
  double pcg_relres = 0.0;
};

struct Work {
  hmle_hmatrix H;
  hmle_hfactor F;
  cudaStream_t st = nullptr, side = nullptr;   // this evaluation's streams (batched use)
  double *d_jacobi = nullptr;                  // its own Jacobi flop counter
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr, done = nullptr;
  double *zdev = nullptr;
  double *zperm = nullptr;         // permuted right-hand side staged for the graph
  bool ready = false;
  cudaGraphExec_t exec = nullptr;  // captured sweep (replayed per theta)
  int graph_kind = -2;             // profiling kind the graph was captured with
  int graph_nev = 0;               // profiling events recorded by one replay
};

// a15: a batch of nz evaluations of one tree in one launch per kernel.  The
// buffers of the nz evaluations (the H-matrix of C, the factor, the
// workspace, flags, results and the Jacobi counter) are carved from one
// allocation with the same layout at a fixed stride, so evaluation z's
// buffers are evaluation 0's shifted by z * stride bytes (FactorArgs::at),
// and every kernel of the sweep serves the whole batch with gridDim.z = nz.
// The batch's sweep is captured once as a CUDA graph and replayed for every
// set of theta (theta lives in each evaluation's device buffer).
struct Group {
  int nz = 0;                       // evaluations of the batch
  int sub = 0;                      // evaluations per launch (a sub-batch)
  char *arena = nullptr;
  int64_t stride = 0;
  std::vector<Work *> w;            // per-evaluation views (own streams for the PCG)
  // per sub-batch: its stream pair, events and captured sweep
  std::vector<cudaStream_t> st, side;
  std::vector<cudaEvent_t> ev_fork, ev_join, done;
  std::vector<cudaGraphExec_t> exec;
  std::vector<int64_t> launches;    // kernel launches of one sub-batch sweep
  unsigned *bar = nullptr;          // grid-barrier words of the batch's persistent sweeps
  double *host = nullptr;           // pinned scalars of the batched PCG (4 + 4 nz)
  int nsub() const { return (nz + sub - 1) / sub; }
};


namespace {

hmle_status fail(hmle_ctx *c, hmle_status s, const std::string &m) {
  if (c) c->err = m;
  return s;
}

hmle_status cuda_fail(hmle_ctx *c, cudaError_t e, const char *where) {
  return fail(c, e == cudaErrorMemoryAllocation ? HMLE_ERR_OOM : HMLE_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                   \
  do {                                                    \
    cudaError_t e__ = (call);                             \
    if (e__ != cudaSuccess) return cuda_fail(ctx, e__, where); \
  } while (0)

bool is_device_ptr(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

template <class T>
cudaError_t upload(cudaStream_t st, T **dst, const std::vector<T> &v, int64_t &bytes) {
  size_t sz = sizeof(T) * std::max<size_t>(v.size(), 1);
  cudaError_t e = cudaMallocAsync((void **)dst, sz, st);
  if (e != cudaSuccess) return e;
  bytes += (int64_t)sz;
  if (!v.empty()) e = cudaMemcpyAsync(*dst, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice, st);
  return e;
}

void free_devplan(cudaStream_t st, DevPlan &d) {
  void *ptrs[] = {d.blocks, d.panels, d.grams, d.gchunks, d.greds, d.lrt, d.aent, d.bent, d.apair, d.bpair,
                  d.lrpairs, d.arow, d.brow, d.arow_ent, d.brow_ent, d.dns, d.dpairs,
                  d.dpair_tr, d.dpair_tc, d.wpan,
                  d.hts, d.urows, d.uents, d.leaf_beg, d.lr_ids, d.dense_ids, d.mv_row0,
                  d.mv_blocks, d.hts_rhs, d.urows_rhs, d.uents_rhs, d.wpan_rhs, d.bh_blocks,
                  d.bupd, d.bents, d.mvt_row0, d.mvt_blocks, d.lr_slot, d.diag, d.ht_rhs0,
                  d.ur_rhs0, d.bh0, d.bupd0, d.hts_mrhs, d.uents_mrhs};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, st);
  d = DevPlan{};
}

// Failures of one evaluation that a batch reports per evaluation (L = -inf)
// without stopping the others: the matrix is not numerically SPD at this
// theta, a low-rank block needed more terms than its capacity, or the mixed
// form's PCG did not reach its tolerance.
bool per_eval_status(hmle_status s) {
  return s == HMLE_OK || s == HMLE_ERR_NOT_SPD || s == HMLE_ERR_RANK_OVERFLOW || s == HMLE_ERR_NOT_CONVERGED;
}

bool theta_ok(const hmle_theta *t) {
  return t && std::isfinite(t->ell) && std::isfinite(t->nu) && std::isfinite(t->sigma2) &&
         std::isfinite(t->tau2) && t->ell > 0 && t->nu > 0 && t->nu <= 20 && t->sigma2 >= 0 &&
         t->tau2 >= 0;
}

void free_hm(cudaStream_t st, hmle_hmatrix *h) {
  if (h->tab) cudaFreeAsync(h->tab, st);
  if (h->uc) cudaFreeAsync(h->uc, st);
  if (h->Cd) cudaFreeAsync(h->Cd, st);
  if (h->rank_c) cudaFreeAsync(h->rank_c, st);
  if (h->cnorm) cudaFreeAsync(h->cnorm, st);
  if (h->thd) cudaFreeAsync(h->thd, st);
  if (h->flags) cudaFreeAsync(h->flags, st);
  h->tab = nullptr; h->uc = nullptr; h->Cd = nullptr; h->rank_c = nullptr; h->cnorm = nullptr;
  h->thd = nullptr; h->flags = nullptr;
}

void free_f(cudaStream_t st, hmle_hfactor *f) {
  void *ptrs[] = {f->D, f->U, f->W, f->ws, f->rank_l, f->kept, f->ldp, f->flags, f->out, f->pcg};
  for (void *p : ptrs)
    if (p) cudaFreeAsync(p, st);
  f->D = f->U = f->W = f->ws = f->pcg = nullptr;
  if (f->pcg_host) cudaFreeHost(f->pcg_host);
  f->pcg_host = nullptr;
  if (f->pcg_init) cudaGraphExecDestroy(f->pcg_init);
  if (f->pcg_iter) cudaGraphExecDestroy(f->pcg_iter);
  f->pcg_init = f->pcg_iter = nullptr;
  f->rank_l = nullptr; f->kept = nullptr; f->ldp = nullptr; f->flags = nullptr; f->out = nullptr;
}

void free_work(Work *w) {
  if (!w) return;
  if (w->exec) cudaGraphExecDestroy(w->exec);
  free_hm(nullptr, &w->H);
  free_f(nullptr, &w->F);
  if (w->zdev) cudaFree(w->zdev);
  if (w->d_jacobi) cudaFree(w->d_jacobi);
  if (w->ev_fork) cudaEventDestroy(w->ev_fork);
  if (w->ev_join) cudaEventDestroy(w->ev_join);
  if (w->done) cudaEventDestroy(w->done);
  if (w->st) cudaStreamDestroy(w->st);
  if (w->side) cudaStreamDestroy(w->side);
  delete w;
}

void free_group(Group *g) {
  if (!g) return;
  for (cudaGraphExec_t x : g->exec)
    if (x) cudaGraphExecDestroy(x);
  for (Work *w : g->w) {
    if (!w) continue;
    // the arena's views are not separate allocations
    w->H.tab = w->H.uc = w->H.Cd = w->H.cnorm = nullptr;
    w->H.rank_c = nullptr; w->H.thd = nullptr; w->H.flags = nullptr;
    w->F.D = w->F.U = w->F.W = w->F.ws = w->F.ldp = w->F.out = nullptr;
    w->F.rank_l = w->F.kept = nullptr; w->F.flags = nullptr;
    w->F.pcg = nullptr;
    w->d_jacobi = nullptr;
    free_work(w);
  }
  if (g->arena) cudaFree(g->arena);
  if (g->bar) cudaFree(g->bar);
  if (g->host) cudaFreeHost(g->host);
  for (cudaEvent_t e : g->ev_fork) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : g->ev_join) if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : g->done) if (e) cudaEventDestroy(e);
  for (cudaStream_t x : g->st) if (x) cudaStreamDestroy(x);
  for (cudaStream_t x : g->side) if (x) cudaStreamDestroy(x);
  delete g;
}

hmle_status alloc_hm(hmle_ctx *ctx, const hmle_tree *t, hmle_hmatrix *h) {
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  h->tree = t;
  CK(cudaMallocAsync(&h->tab, sizeof(double) * kTableWords, st), "alloc table");
  CK(cudaMallocAsync(&h->uc, sizeof(double) * std::max<int64_t>(P.uc_words, 1), st), "alloc C factors");
  CK(cudaMallocAsync(&h->Cd, sizeof(double) * std::max<int64_t>(P.dense_words, 1), st), "alloc dense near field");
  CK(cudaMallocAsync(&h->rank_c, sizeof(int32_t) * std::max<size_t>(P.blocks.size(), 1), st), "alloc ranks");
  CK(cudaMallocAsync(&h->cnorm, sizeof(double) * std::max<size_t>(P.blocks.size(), 1), st), "alloc norms");
  CK(cudaMemsetAsync(h->cnorm, 0, sizeof(double) * std::max<size_t>(P.blocks.size(), 1), st), "memset");
  CK(cudaMallocAsync(&h->thd, sizeof(ThetaDev), st), "alloc theta");
  CK(cudaMallocAsync(&h->flags, sizeof(int), st), "alloc flags");
  CK(cudaMemsetAsync(h->rank_c, 0, sizeof(int32_t) * std::max<size_t>(P.blocks.size(), 1), st), "memset");
  return HMLE_OK;
}

hmle_status alloc_f(hmle_ctx *ctx, const hmle_tree *t, hmle_hfactor *f) {
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  CK(cudaMallocAsync(&f->D, sizeof(double) * std::max<int64_t>(P.dense_words, 1), st), "alloc dense pool");
  CK(cudaMallocAsync(&f->U, sizeof(double) * std::max<int64_t>(P.u_words, 1), st), "alloc U pool");
  CK(cudaMallocAsync(&f->W, sizeof(double) * std::max<int64_t>(P.w_words, 1), st), "alloc W panels");
  CK(cudaMallocAsync(&f->ws, sizeof(double) * std::max<int64_t>(P.ws_max, 1), st), "alloc workspace");
  CK(cudaMallocAsync(&f->rank_l, sizeof(int32_t) * std::max<size_t>(P.blocks.size(), 1), st), "alloc ranks");
  CK(cudaMallocAsync(&f->kept, sizeof(int32_t) * std::max<size_t>(P.lrt.size(), 1), st), "alloc kept");
  CK(cudaMallocAsync(&f->ldp, sizeof(double) * P.nleaf, st), "alloc logdet");
  CK(cudaMallocAsync(&f->flags, sizeof(int), st), "alloc flags");
  CK(cudaMallocAsync(&f->out, sizeof(double) * 2, st), "alloc out");
  return HMLE_OK;
}

// assemble into h (buffers allocated)
hmle_status do_assemble(hmle_ctx *ctx, const hmle_tree *t, const hmle_theta *th, hmle_hmatrix *h) {
  cudaStream_t st = ctx->st;
  cudaGetLastError();  // errors of earlier, unrelated runtime calls are not ours
  const Plan &P = t->plan;
  h->th = *th;
  ThetaDev td{1.0 / th->ell, th->sigma2, th->tau2, th->nu};
  CK(cudaMemcpyAsync(h->thd, &td, sizeof(td), cudaMemcpyHostToDevice, st), "theta upload");
  CK(cudaMemsetAsync(h->flags, 0, sizeof(int), st), "memset flags");
  launch_matern_table(st, th->nu, h->tab);
  AsmArgs A{};
  A.blocks = t->dp.blocks;
  A.lr_ids = t->dp.lr_ids;
  A.xyz = t->T.xyz;
  A.n = t->n;
  A.d = t->d;
  A.tab = h->tab;
  A.inv_ell = 1.0 / th->ell;
  A.sigma2 = th->sigma2;
  A.tau2 = th->tau2;
  A.eps = t->opts.aca_eps;
  A.kc = P.kc;
  A.uc = h->uc;
  A.rank_c = h->rank_c;
  A.cnorm = h->cnorm;
  A.flags = h->flags;
  A.fixed_k = t->opts.fixed_rank;
  launch_aca(st, A, (int)t->lr_ids.size());
  launch_assemble_dense(st, A, t->dp.dense_ids, (int)t->dense_ids.size(), P.b, h->Cd);
  CK(cudaGetLastError(), "assemble launch");
  return HMLE_OK;
}

// Truncation floor of the mixed factors: the tensor-core products carry
// their operands to 24 bits (HMLE_MIXED_FP32, three BF16 slices) or 16 bits
// (HMLE_MIXED_BF16, two slices) and leave noise near 1e-7 or 1e-5 of a
// block's norm in a Schur complement.
constexpr double kMixedTruncEps[3] = {0.0, 1e-7, 1e-5};
inline bool is_mixed(int32_t precision) { return precision == HMLE_MIXED_FP32 || precision == HMLE_MIXED_BF16; }
constexpr int kAssemblyLaunches = 3;      // Matern table, ACA, dense near field of one assembly

FactorArgs make_fargs(const hmle_tree *t, const hmle_hmatrix *h, hmle_hfactor *f) {
  const Plan &P = t->plan;
  const DevPlan &d = t->dp;
  FactorArgs F{};
  F.blocks = d.blocks; F.panels = d.panels; F.grams = d.grams; F.lrt = d.lrt;
  F.gchunks = d.gchunks; F.greds = d.greds;
  F.aent = d.aent; F.bent = d.bent; F.apair = d.apair; F.bpair = d.bpair;
  F.lrpairs = d.lrpairs; F.arow = d.arow; F.brow = d.brow; F.arow_ent = d.arow_ent;
  F.brow_ent = d.brow_ent; F.dns = d.dns; F.dpairs = d.dpairs; F.wpan = d.wpan;
  F.dpair_tr = d.dpair_tr; F.dpair_tc = d.dpair_tc;
  F.hts = d.hts; F.urows = d.urows; F.uents = d.uents; F.leaf_beg = d.leaf_beg;
  F.D = f->D; F.uc = h->uc; F.Cd = h->Cd; F.rank_c = h->rank_c; F.cnorm = h->cnorm; F.U = f->U; F.W = f->W; F.ws = f->ws;
  F.rank_l = f->rank_l; F.kept = f->kept; F.logdet_parts = f->ldp; F.flags = f->flags;
  F.xyz = t->T.xyz; F.n = t->n; F.d = t->d; F.tab = h->tab; F.th = h->thd;
  F.eps = t->opts.aca_eps; F.seed = t->opts.seed;
  F.b = P.b; F.kcap = P.kcap; F.kc = P.kc; F.r = P.r;
  F.osamp = t->opts.oversample;
  F.mixed = is_mixed(t->opts.precision) ? t->opts.precision : 0;
  F.fixed_k = t->opts.fixed_rank;
  F.nz = 1;          // one evaluation; a batch sets nz and the stride of its buffers
  F.zstride = 0;
  // The low-precision products leave noise of about 1e-7 (FP32-class) or
  // 1e-5 (16-bit) of |C_T| in a Schur complement; truncating below that would
  // keep noise as rank.  The mixed factor is truncated at max(eps, floor);
  // the accuracy of the quadratic form comes from the FP64 operator of the
  // PCG (ACA at eps).
  if (F.mixed) F.eps = std::max(F.eps, kMixedTruncEps[F.mixed]);
  return F;
}

// a14: in the mixed form the quadratic form of the fused forward solve carries
// the FP32 rounding of the factor; it is replaced by b^T x with C x = b solved
// by PCG (FP64 operator, the mixed factor as preconditioner).  zdev: Z in the
// caller's order, on the device.
hmle_status mixed_prepare(hmle_ctx *ctx, const hmle_tree *t, const hmle_hmatrix *h, hmle_hfactor *f,
                          const double *zdev, PcgRun &R) {
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  const int nlr = (int)t->lr_ids.size();
  int hmax = 1;
  for (int K = 0; K < P.nleaf; ++K) hmax = std::max(hmax, P.bh0[K + 1] - P.bh0[K]);
  if (!f->pcg) {
    const int64_t words = t->n + pcg_words(t->n, nlr, P.kc, hmax * P.kcap) + 2;
    cudaError_t e = cudaMallocAsync(&f->pcg, sizeof(double) * words, st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pcg workspace");
  }
  if (!f->pcg_host) {
    cudaError_t e = cudaMallocHost(&f->pcg_host, 4 * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "pcg host scalars");
  }
  double *b = f->pcg;
  launch_permute_in(st, zdev, t->T.perm, t->n, b);
  AsmArgs A{};
  A.blocks = t->dp.blocks; A.lr_ids = t->dp.lr_ids; A.xyz = t->T.xyz; A.n = t->n; A.d = t->d;
  A.tab = h->tab; A.inv_ell = 1.0 / h->th.ell; A.sigma2 = h->th.sigma2; A.tau2 = h->th.tau2;
  A.kc = P.kc; A.uc = h->uc; A.rank_c = h->rank_c; A.cnorm = h->cnorm; A.flags = h->flags;
  A.thd = h->thd; A.Cd = h->Cd; A.b = P.b;
  FactorArgs Fs = make_fargs(t, h, f);
  Fs.hts = t->dp.hts_rhs;
  Fs.urows = t->dp.urows_rhs;
  Fs.uents = t->dp.uents_rhs;
  const PanelDesc &rp = P.panels[P.rhs_panel];
  R = PcgRun{};
  R.st = st; R.A = A; R.n_lr = nlr;
  R.L = CmvLists{P.nleaf, t->dp.leaf_beg, t->dp.mv_row0, t->dp.mv_blocks, t->dp.mvt_row0,
                 t->dp.mvt_blocks, t->dp.lr_slot};
  R.Fs = Fs; R.PL = &P; R.wpan_rhs = t->dp.wpan_rhs; R.bh_blocks = t->dp.bh_blocks;
  R.bupd = t->dp.bupd; R.bents = t->dp.bents; R.panel = f->W + rp.off; R.b = b; R.n = t->n;
  R.tol = t->opts.pcg_tol; R.maxit = t->opts.pcg_max_iter; R.pool = f->pcg + t->n;
  R.host = f->pcg_host;
  // the persistent sweeps (one cooperative launch each) when the device has
  // them; the CUDA graphs otherwise replay the launch-by-launch sweeps
  R.SP = t->coop ? &t->sp : nullptr;
  R.bar = reinterpret_cast<unsigned *>(f->pcg + t->n + pcg_words(t->n, nlr, P.kc, hmax * P.kcap));
  R.g_init = (t->graphs && !R.SP) ? &f->pcg_init : nullptr;
  R.g_iter = (t->graphs && !R.SP) ? &f->pcg_iter : nullptr;
  return HMLE_OK;
}

hmle_status mixed_result(hmle_ctx *ctx, const hmle_tree *t, hmle_hfactor *f, const PcgRun &R) {
  if (R.timed_out) return fail(ctx, HMLE_ERR_TIMEOUT, "PCG: a barrier wait of the persistent sweep ran out");
  f->quad = R.q;
  f->pcg_iters = R.it;
  f->pcg_relres = R.rel;
  f->has_rhs = true;
  if (!(R.rel <= t->opts.pcg_tol) || !std::isfinite(R.q))
    return fail(ctx, HMLE_ERR_NOT_CONVERGED, "PCG: relative residual above pcg_tol after pcg_max_iter");
  return HMLE_OK;
}

// a14: in the mixed form the quadratic form of the fused forward solve carries
// the FP32 rounding of the factor; it is replaced by b^T x with C x = b solved
// by PCG (FP64 operator, the mixed factor as preconditioner).  zdev: Z in the
// caller's order, on the device.
hmle_status mixed_quad(hmle_ctx *ctx, const hmle_tree *t, const hmle_hmatrix *h, hmle_hfactor *f,
                       const double *zdev) {
  PcgRun R;
  hmle_status s = mixed_prepare(ctx, t, h, f, zdev, R);
  if (s != HMLE_OK) return s;
  cudaError_t e = pcg_quad(R);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "pcg");
  return mixed_result(ctx, t, f, R);
}

// The launch sequence of one factorisation (sweep + finalize) on stream st.
int64_t launch_sweep(hmle_ctx *ctx, const hmle_tree *t, const hmle_hmatrix *h, hmle_hfactor *f,
                     Prof *prof) {
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  FactorArgs F = make_fargs(t, h, f);
  F.jacobi_flops = ctx->d_jacobi;
  cudaMemsetAsync(f->flags, 0, sizeof(int), st);
  cudaMemsetAsync(f->rank_l, 0, sizeof(int32_t) * std::max<size_t>(P.blocks.size(), 1), st);
  cudaMemsetAsync(ctx->d_jacobi, 0, sizeof(double), st);
  int64_t nk = 2;  // permutation, finalize
  for (int K = 0; K < P.nleaf; ++K)
    nk += launch_step(st, ctx->side, ctx->ev_fork, ctx->ev_join, F, P.steps[K], K, P, prof);
  const PanelDesc &rp = P.panels[P.rhs_panel];
  launch_finalize(st, f->ldp, P.nleaf, f->W + rp.off, t->n, f->out);
  return nk;
}

hmle_status launch_factor_async(hmle_ctx *ctx, const hmle_tree *t, const hmle_hmatrix *h,
                                const double *zdev, hmle_hfactor *f, Work *w) {
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  f->h = h;
  const PanelDesc &rp = P.panels[P.rhs_panel];
  launch_permute_in(st, zdev, t->T.perm, t->n, f->W + rp.off);
  f->has_rhs = true;
  if (!w) {
    f->launches = launch_sweep(ctx, t, h, f, nullptr) + kAssemblyLaunches;
  } else if (!w->exec || w->graph_kind != -1) {
    if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
    int64_t nk = launch_sweep(ctx, t, h, f, nullptr);
    cudaError_t e = cudaStreamEndCapture(st, &g);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
    e = cudaGraphInstantiate(&w->exec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { w->exec = nullptr; return cuda_fail(ctx, e, "graph instantiate"); }
    w->graph_kind = -1;
    w->graph_nev = 0;
    f->launches = nk + kAssemblyLaunches;
  }
  if (w) CK(cudaGraphLaunch(w->exec, st), "graph launch");
  // no copy to host here: host_out is pageable, and a device-to-pageable copy
  // returns only when it has completed, which would make the caller wait for
  // this evaluation before it can launch the next one
  return HMLE_OK;
}

hmle_status finish_factor(hmle_ctx *ctx, const hmle_tree *t, const hmle_hmatrix *h, hmle_hfactor *f) {
  cudaStream_t st = ctx->st;
  CK(cudaStreamSynchronize(st), "factor sync");
  CK(cudaMemcpyAsync(f->host_out, f->out, 2 * sizeof(double), cudaMemcpyDeviceToHost, st), "result copy");
  CK(cudaMemcpyAsync(&f->host_flags[0], f->flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
  CK(cudaMemcpyAsync(&f->host_flags[1], h->flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
  CK(cudaStreamSynchronize(st), "result sync");
  f->logdet = f->host_out[0];
  f->quad = f->host_out[1];
  int fl = f->host_flags[0] | f->host_flags[1];
  if (fl & kFlagTimeout) return fail(ctx, HMLE_ERR_TIMEOUT, "a tensor-core product did not complete in time");
  if (fl & kFlagNotSpd) return fail(ctx, HMLE_ERR_NOT_SPD, "non-positive pivot in a diagonal leaf");
  if (fl & kFlagRankOverflow)
    return fail(ctx, HMLE_ERR_RANK_OVERFLOW, "a low-rank block needed more than max_rank terms");
  if (!std::isfinite(f->logdet) || !std::isfinite(f->quad))
    return fail(ctx, HMLE_ERR_NOT_SPD, "non-finite log-determinant or quadratic form");
  (void)t; (void)h;
  return HMLE_OK;
}

hmle_status do_factor(hmle_ctx *ctx, const hmle_tree *t, const hmle_hmatrix *h,
                      const double *zdev, hmle_hfactor *f, Work *w = nullptr) {
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  f->h = h;
  const PanelDesc &rp = P.panels[P.rhs_panel];
  if (zdev) {
    launch_permute_in(st, zdev, t->T.perm, t->n, f->W + rp.off);
    f->has_rhs = true;
  } else {
    CK(cudaMemsetAsync(f->W + rp.off, 0, sizeof(double) * t->n, st), "memset rhs");
    f->has_rhs = false;
  }
  Prof *prof = ctx->prof.kind >= 0 ? &ctx->prof : nullptr;
  int nev = 0;
  if (w) {
    // replay (capturing first) the graph of the sweep
    if (!w->exec || w->graph_kind != ctx->prof.kind) {
      if (w->exec) { cudaGraphExecDestroy(w->exec); w->exec = nullptr; }
      cudaGraph_t g = nullptr;
      if (prof) prof->used = 0;
      CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "begin capture");
      int64_t nk = launch_sweep(ctx, t, h, f, prof);
      cudaError_t e = cudaStreamEndCapture(st, &g);
      if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
      e = cudaGraphInstantiate(&w->exec, g, 0);
      cudaGraphDestroy(g);
      if (e != cudaSuccess) { w->exec = nullptr; return cuda_fail(ctx, e, "graph instantiate"); }
      w->graph_kind = ctx->prof.kind;
      w->graph_nev = prof ? prof->used : 0;
      f->launches = nk + kAssemblyLaunches;
    }
    CK(cudaGraphLaunch(w->exec, st), "graph launch");
    nev = w->graph_nev;
  } else {
    if (prof) prof->used = 0;
    f->launches = launch_sweep(ctx, t, h, f, prof) + kAssemblyLaunches;
    nev = prof ? prof->used : 0;
  }
  CK(cudaGetLastError(), "factor launch");
  double out[2];
  int flags[2];
  CK(cudaMemcpyAsync(out, f->out, sizeof(out), cudaMemcpyDeviceToHost, st), "result copy");
  CK(cudaMemcpyAsync(&flags[0], f->flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
  CK(cudaMemcpyAsync(&flags[1], h->flags, sizeof(int), cudaMemcpyDeviceToHost, st), "flag copy");
  CK(cudaStreamSynchronize(st), "factor sync");
  f->logdet = out[0];
  f->quad = out[1];
  if (prof) {
    prof_collect(prof, nev);
    if (prof->failed)
      ctx->err = "profiler: " + std::to_string(prof->failed) + " event pairs unreadable (" +
                 cudaGetErrorString((cudaError_t)prof->first_err) + "), " + std::to_string(nev) +
                 " events recorded";
    std::vector<int32_t> rc(P.blocks.size()), rl(P.blocks.size()), kp(std::max<size_t>(P.lrt.size(), 1));
    double jf = 0.0;
    CK(cudaMemcpy(rc.data(), h->rank_c, sizeof(int32_t) * rc.size(), cudaMemcpyDeviceToHost), "ranks");
    CK(cudaMemcpy(rl.data(), f->rank_l, sizeof(int32_t) * rl.size(), cudaMemcpyDeviceToHost), "ranks");
    CK(cudaMemcpy(kp.data(), f->kept, sizeof(int32_t) * kp.size(), cudaMemcpyDeviceToHost), "kept");
    CK(cudaMemcpy(&jf, ctx->d_jacobi, sizeof(double), cudaMemcpyDeviceToHost), "jacobi");
    prof->flops += tally_flops(P, prof->kind, rc, rl, kp, t->opts.oversample, jf);
  }
  int fl = flags[0] | flags[1];
  if (fl & kFlagTimeout) return fail(ctx, HMLE_ERR_TIMEOUT, "a tensor-core product did not complete in time");
  if (fl & kFlagNotSpd) return fail(ctx, HMLE_ERR_NOT_SPD, "non-positive pivot in a diagonal leaf");
  if (fl & kFlagRankOverflow)
    return fail(ctx, HMLE_ERR_RANK_OVERFLOW, "a low-rank block needed more than max_rank terms");
  if (!std::isfinite(out[0]) || !std::isfinite(out[1]))
    return fail(ctx, HMLE_ERR_NOT_SPD, "non-finite log-determinant or quadratic form");
  return HMLE_OK;
}

hmle_status rank_stats(hmle_ctx *ctx, const hmle_tree *t, const int32_t *dranks, int *maxr,
                       double *meanr) {
  std::vector<int32_t> rk(t->plan.blocks.size());
  if (rk.empty()) { *maxr = 0; *meanr = 0; return HMLE_OK; }
  CK(cudaMemcpyAsync(rk.data(), dranks, sizeof(int32_t) * rk.size(), cudaMemcpyDeviceToHost, ctx->st), "ranks");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  int mx = 0; double s = 0; int c = 0;
  for (int32_t x : t->lr_ids) { mx = std::max(mx, rk[x]); s += rk[x]; ++c; }
  *maxr = mx;
  *meanr = c ? s / c : 0.0;
  return HMLE_OK;
}

hmle_status stage_vec(hmle_ctx *ctx, const double *src, int64_t n, double **dev, bool *owned) {
  if (is_device_ptr(src)) { *dev = const_cast<double *>(src); *owned = false; return HMLE_OK; }
  CK(cudaMallocAsync(dev, sizeof(double) * std::max<int64_t>(n, 1), ctx->st), "alloc vector");
  CK(cudaMemcpyAsync(*dev, src, sizeof(double) * n, cudaMemcpyHostToDevice, ctx->st), "copy vector");
  *owned = true;
  return HMLE_OK;
}

// The H-matrix plan of a tree from its block tree and options: the schedule
// of the leaf sweep (Sec. 2, H-Cholesky) with the storage of every block at
// the tree's rank capacities, uploaded to the device.  A tree derived with
// other capacities (rank-overflow retry) shares the cluster tree and runs
// this again.
hmle_status plan_tree(hmle_ctx *ctx, hmle_tree *t) {
  cudaStream_t st = ctx->st;
  const hmle_opts &o = t->opts;
  const int depth = tree_depth(t->n, o.leaf_size);
  const std::vector<int32_t> &cb = t->cb, &ce = t->ce;
  std::vector<int4> blocks = t->blocks0;
  const int64_t n = t->n;
  const int d = t->d;
  const int kc = o.max_rank + 16 <= 64 ? o.max_rank + 16 : 64;  // ACA capacity for C
  if (!o.leaf_lowrank)  // leaf x leaf admissible blocks are kept dense (exact)
    for (int4 &q : blocks)
      if (q.w == kLowRank && q.x == depth) q.w = kDense;
  std::string err = build_plan(t->plan, (int32_t)n, d, o.leaf_size, depth, cb, ce, blocks, o.max_rank, kc,
                   o.max_rank + o.oversample, 1);
  if (!err.empty()) return fail(ctx, HMLE_ERR_INVALID_ARG, "planner: " + err);
  const Plan &P = t->plan;
  for (size_t x = 0; x < P.blocks.size(); ++x)
    (P.blocks[x].kind == kLowRank ? t->lr_ids : t->dense_ids).push_back((int32_t)x);
  std::vector<int2> dtr(P.dpairs.size()), dtc(P.dpairs.size());
  for (const DenseTarget &dt : P.dns) {
    const BlockDesc &T = P.blocks[dt.blk];
    for (int q = dt.p0; q < dt.p1; ++q) {
      dtr[q] = make_int2(T.rbeg, T.rend);
      dtc[q] = make_int2(T.cbeg, T.cend);
    }
  }
  std::vector<int32_t> leaf_beg(P.nleaf + 1);
  for (int K = 0; K < P.nleaf; ++K) leaf_beg[K] = cb[(1 << depth) - 1 + K];
  leaf_beg[P.nleaf] = (int32_t)n;
  DevPlan &dp = t->dp;
  cudaError_t e = cudaSuccess;
#define UP(f, v) if (e == cudaSuccess) e = upload(st, &dp.f, v, dp.bytes)
  UP(blocks, P.blocks); UP(panels, P.panels); UP(grams, P.grams); UP(lrt, P.lrt);
  UP(gchunks, P.gchunks); UP(greds, P.greds);
  UP(aent, P.aent); UP(bent, P.bent); UP(apair, P.apair); UP(bpair, P.bpair);
  UP(lrpairs, P.lrpairs); UP(arow, P.arow); UP(brow, P.brow); UP(arow_ent, P.arow_ent);
  UP(brow_ent, P.brow_ent); UP(dns, P.dns); UP(dpairs, P.dpairs); UP(wpan, P.wpan);
  UP(dpair_tr, dtr); UP(dpair_tc, dtc);
  UP(hts, P.hts); UP(urows, P.urows); UP(uents, P.uents); UP(leaf_beg, leaf_beg);
  UP(lr_ids, t->lr_ids); UP(dense_ids, t->dense_ids);
  UP(mv_row0, P.mv_row0); UP(mv_blocks, P.mv_blocks);
  UP(hts_rhs, P.hts_rhs); UP(urows_rhs, P.urows_rhs); UP(uents_rhs, P.uents_rhs);
  UP(bh_blocks, P.bh_blocks); UP(bupd, P.bupd); UP(bents, P.bents);
  UP(mvt_row0, P.mvt_row0); UP(mvt_blocks, P.mvt_blocks);
  UP(diag, P.diag_of_leaf); UP(ht_rhs0, P.ht_rhs0); UP(ur_rhs0, P.ur_rhs0); UP(bh0, P.bh0);
  UP(bupd0, P.bupd0);
  {
    std::vector<int32_t> slot(std::max<size_t>(P.blocks.size(), 1), -1);
    for (size_t q = 0; q < t->lr_ids.size(); ++q) slot[t->lr_ids[q]] = (int32_t)q;
    UP(lr_slot, slot);
  }
  {
    std::vector<int32_t> wr(1, P.rhs_panel);
    UP(wpan_rhs, wr);
  }
  {  // forward lists of the multi-vector sweep: a task's coupling vector at
     // kcap doubles per task of its leaf instead of its place in the factor's
     // workspace, so that each vector needs only the largest leaf's share
    std::vector<HTask> hc = P.hts_rhs;
    std::vector<UpdEntry> uc = P.uents_rhs;
    int64_t hw = 1;
    bool ok = true;
    for (int K = 0; K < P.nleaf && ok; ++K) {
      std::map<int64_t, int64_t> slot;
      for (int q = P.ht_rhs0[K]; q < P.ht_rhs0[K + 1]; ++q) {
        const int64_t c = (int64_t)(q - P.ht_rhs0[K]) * P.kcap;
        slot[hc[q].hoff] = c;
        hc[q].hoff = c;
      }
      hw = std::max<int64_t>(hw, (int64_t)(P.ht_rhs0[K + 1] - P.ht_rhs0[K]) * P.kcap);
      hw = std::max<int64_t>(hw, (int64_t)(P.bh0[K + 1] - P.bh0[K]) * P.kcap);
      for (int r = P.ur_rhs0[K]; r < P.ur_rhs0[K + 1] && ok; ++r)
        for (int q = P.urows_rhs[r].e0; q < P.urows_rhs[r].e1; ++q) {
          if (uc[q].hoff < 0) continue;
          auto it = slot.find(uc[q].hoff);
          if (it == slot.end()) { ok = false; break; }
          uc[q].hoff = it->second;
        }
    }
    if (!ok) return fail(ctx, HMLE_ERR_INVALID_ARG, "planner: a forward update without its leaf's task");
    t->mrhs_h = hw;
    UP(hts_mrhs, hc);
    UP(uents_mrhs, uc);
  }
#undef UP
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "plan upload");
  {
    const DevPlan &d = t->dp;
    t->sp = SolvePlan{P.nleaf, d.diag, d.ht_rhs0, d.ur_rhs0, d.hts_rhs, d.urows_rhs, d.uents_rhs,
                      d.bh0, d.bupd0, d.bh_blocks, d.bupd, d.bents};
    t->spm = t->sp;
    t->spm.hts = d.hts_mrhs;
    t->spm.uents = d.uents_mrhs;
    int coop = 0;
    cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, ctx->dev);
    t->coop = coop != 0;
  }
  return HMLE_OK;
}

// A tree on the same points and cluster tree as src with other options
// (rank capacities, precision, accuracy): only the plan is made again.  The
// derived tree borrows src's cluster tree and must be destroyed first.
hmle_status derive_tree(hmle_ctx *ctx, const hmle_tree *src, const hmle_opts &o, hmle_tree **out) {
  hmle_tree *t = new (std::nothrow) hmle_tree();
  if (!t) return fail(ctx, HMLE_ERR_OOM, "derived tree");
  t->ctx = ctx; t->n = src->n; t->d = src->d; t->opts = o; t->graphs = src->graphs;
  t->T = src->T;
  t->owns_T = false;
  t->blocks0 = src->blocks0; t->cb = src->cb; t->ce = src->ce;
  hmle_status s = plan_tree(ctx, t);
  if (s != HMLE_OK) { hmle_tree_destroy(t); return s; }
  *out = t;
  return HMLE_OK;
}

}  // namespace

extern "C" {

// stream of a context, for the other translation units of the library
__attribute__((visibility("hidden"))) cudaStream_t hmle_internal_ctx_stream(const hmle_ctx *c) {
  return c ? c->st : nullptr;
}

// device that owns a context's stream, and the context's error path, for the
// other translation units of the library
__attribute__((visibility("hidden"))) int hmle_internal_ctx_device(const hmle_ctx *c) {
  return c ? c->dev : -1;
}
__attribute__((visibility("hidden"))) hmle_status hmle_internal_ctx_fail(hmle_ctx *c, hmle_status s,
                                                                        const char *msg) {
  return fail(c, s, msg ? msg : "");
}

hmle_status hmle_opts_default(hmle_opts *o) {
  if (!o) return HMLE_ERR_INVALID_ARG;
  o->leaf_size = 64;
  o->eta = 2.0;
  o->aca_eps = 1e-8;
  o->max_rank = 32;
  o->oversample = 8;
  o->precision = HMLE_FP64;
  o->pcg_tol = 1e-10;
  o->pcg_max_iter = 50;
  o->seed = 0x5eed;
  o->leaf_lowrank = 0;
  o->fixed_rank = 0;
  o->batch_size = 2;
  return HMLE_OK;
}

hmle_status hmle_fit_opts_default(hmle_fit_opts *o) {
  if (!o) return HMLE_ERR_INVALID_ARG;
  o->ftol = 1e-4;
  o->xtol = 1e-4;
  o->max_iter = 400;
  for (int i = 0; i < 4; ++i) o->step[i] = 1.0;
  return HMLE_OK;
}

hmle_status hmle_ctx_create(hmle_ctx **out, void *stream) {
  if (!out) return HMLE_ERR_INVALID_ARG;
  hmle_ctx *c = new (std::nothrow) hmle_ctx();
  if (!c) return HMLE_ERR_OOM;
  cudaError_t e = cudaGetDevice(&c->dev);
  if (e == cudaSuccess && stream) {
    c->st = (cudaStream_t)stream;
  } else if (e == cudaSuccess) {
    e = cudaStreamCreateWithFlags(&c->st, cudaStreamNonBlocking);
    c->own = true;
  }
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->side, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaMalloc(&c->d_jacobi, sizeof(double));
  if (e != cudaSuccess) {
    delete c;
    return HMLE_ERR_CUDA;
  }
  *out = c;
  return HMLE_OK;
}

void hmle_ctx_destroy(hmle_ctx *c) {
  if (!c) return;
  if (c->ev_fork) cudaEventDestroy(c->ev_fork);
  if (c->ev_join) cudaEventDestroy(c->ev_join);
  if (c->side) cudaStreamDestroy(c->side);
  for (cudaEvent_t ev : c->prof.ev) cudaEventDestroy(ev);
  if (c->d_jacobi) cudaFree(c->d_jacobi);
  if (c->own && c->st) cudaStreamDestroy(c->st);
  delete c;
}

const char *hmle_last_error(const hmle_ctx *c) { return c ? c->err.c_str() : "null context"; }

hmle_status hmle_build_tree(hmle_ctx *ctx, const double *locs, int64_t n, int32_t d,
                            const hmle_opts *opts_in, hmle_tree **out) {
  if (!ctx || !locs || !out) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  hmle_opts o;
  if (opts_in) o = *opts_in; else hmle_opts_default(&o);
  if (n < 2 || n > (1LL << 30)) return fail(ctx, HMLE_ERR_INVALID_ARG, "n out of range");
  if (d != 2 && d != 3) return fail(ctx, HMLE_ERR_INVALID_ARG, "d must be 2 or 3");
  if (o.leaf_size < 8 || o.leaf_size > kMaxLeaf || (o.leaf_size % 16) != 0)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "leaf_size must be a multiple of 16 in [16, 128]");
  if (!(o.eta > 0) || !(o.aca_eps > 0) || !(o.aca_eps < 1))
    return fail(ctx, HMLE_ERR_INVALID_ARG, "eta > 0 and 0 < aca_eps < 1 required");
  if (o.max_rank < 8 || o.max_rank > 64 || (o.max_rank % 8) != 0)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "max_rank must be a multiple of 8 in [8, 64]");
  if (o.fixed_rank < 0 || o.fixed_rank > o.max_rank)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "fixed_rank must be in [0, max_rank]");
  if (o.batch_size < 1 || o.batch_size > 64)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "batch_size must be in [1, 64]");
  if (o.oversample < 4 || o.max_rank + o.oversample > 64)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "oversample >= 4 and max_rank + oversample <= 64");
  if (o.precision != HMLE_FP64 && !is_mixed(o.precision))
    return fail(ctx, HMLE_ERR_INVALID_ARG, "precision");
  if (is_mixed(o.precision) && !(o.pcg_tol > 0.0 && o.pcg_max_iter >= 1))
    return fail(ctx, HMLE_ERR_INVALID_ARG, "pcg_tol / pcg_max_iter");
  static bool smem_ok = false;
  if (!smem_ok) {
    int rc = factor_smem_setup(kMaxLeaf, 64);
    if (rc) return fail(ctx, HMLE_ERR_CUDA, "cudaFuncSetAttribute failed");
    smem_ok = true;
  }
  cudaStream_t st = ctx->st;
  // cluster ranges (pure integer, host)
  const int depth = tree_depth(n, o.leaf_size);
  if (depth > kMaxLevels - 2) return fail(ctx, HMLE_ERR_INVALID_ARG, "tree too deep");
  std::vector<int32_t> cb, ce;
  cluster_ranges(n, depth, cb, ce);
  hmle_tree *t = new (std::nothrow) hmle_tree();
  if (!t) return HMLE_ERR_OOM;
  t->ctx = ctx; t->n = n; t->d = d; t->opts = o;
  {  // HMLE_GRAPHS=0 launches the sweep kernel by kernel (for profilers)
    const char *g = std::getenv("HMLE_GRAPHS");
    t->graphs = !(g && g[0] == '0');
  }
  double *rows = nullptr;
  bool owned = false;
  hmle_status s = stage_vec(ctx, locs, n * d, &rows, &owned);
  if (s != HMLE_OK) { delete t; return s; }
  std::vector<int4> blocks;
  std::string err = tree_build_device(st, rows, n, d, depth, cb, ce, o.eta, t->T, blocks);
  if (owned) cudaFreeAsync(rows, st);
  if (!err.empty()) {
    hmle_tree_destroy(t);
    return fail(ctx, err.find("non-finite") != std::string::npos ? HMLE_ERR_INVALID_ARG : HMLE_ERR_CUDA, err);
  }
  t->blocks0 = std::move(blocks);
  t->cb = std::move(cb);
  t->ce = std::move(ce);
  s = plan_tree(ctx, t);
  if (s != HMLE_OK) { hmle_tree_destroy(t); return s; }
  *out = t;
  return HMLE_OK;
}

void hmle_tree_destroy(hmle_tree *t) {
  if (!t) return;
  // the context may already be gone: free synchronously on the legacy stream
  cudaStream_t st = nullptr;
  cudaDeviceSynchronize();
  if (t->work) {
    if (t->work->exec) cudaGraphExecDestroy(t->work->exec);
    free_hm(st, &t->work->H);
    free_f(st, &t->work->F);
    if (t->work->zdev) cudaFreeAsync(t->work->zdev, st);
    delete t->work;
  }
  for (Work *w : t->pool) free_work(w);
  for (Group *g : t->groups) free_group(g);
  free_devplan(st, t->dp);
  if (t->owns_T) {
    if (t->T.xyz) cudaFreeAsync(t->T.xyz, st);
    if (t->T.perm) cudaFreeAsync(t->T.perm, st);
    if (t->T.box) cudaFreeAsync(t->T.box, st);
  }
  cudaStreamSynchronize(st);
  delete t;
}

hmle_status hmle_tree_set_batch_size(hmle_tree *t, int32_t batch_size) {
  if (!t || batch_size < 1 || batch_size > 64) return HMLE_ERR_INVALID_ARG;
  t->opts.batch_size = batch_size;
  return HMLE_OK;
}

hmle_status hmle_tree_get_info(const hmle_tree *t, hmle_tree_info *info) {
  if (!t || !info) return HMLE_ERR_INVALID_ARG;
  const Plan &P = t->plan;
  info->n = t->n;
  info->d = t->d;
  info->depth = P.depth;
  info->n_leaves = P.nleaf;
  info->n_dense = (int32_t)P.n_dense_blocks;
  info->n_lowrank = (int32_t)P.n_lr_blocks;
  info->dense_words = P.dense_words;
  info->lowrank_words = P.uc_words + P.u_words + P.w_words;
  info->device_bytes = t->dp.bytes + (int64_t)t->n * (3 * 8 + 4);
  return HMLE_OK;
}

hmle_status hmle_tree_permutation(const hmle_tree *t, int32_t *perm) {
  if (!t || !perm) return HMLE_ERR_INVALID_ARG;
  hmle_ctx *ctx = t->ctx;
  CK(cudaMemcpyAsync(perm, t->T.perm, sizeof(int32_t) * t->n, cudaMemcpyDeviceToHost, ctx->st), "perm copy");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  return HMLE_OK;
}

hmle_status hmle_assemble(hmle_ctx *ctx, const hmle_tree *t, const hmle_theta *th,
                          hmle_hmatrix **out) {
  if (!ctx || !t || !out) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!theta_ok(th)) return fail(ctx, HMLE_ERR_INVALID_ARG, "theta out of range");
  hmle_hmatrix *h = new (std::nothrow) hmle_hmatrix();
  if (!h) return HMLE_ERR_OOM;
  hmle_status s = alloc_hm(ctx, t, h);
  if (s == HMLE_OK) s = do_assemble(ctx, t, th, h);
  if (s == HMLE_OK) {
    int fl = 0;
    cudaError_t e = cudaMemcpyAsync(&fl, h->flags, sizeof(int), cudaMemcpyDeviceToHost, ctx->st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->st);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "assemble");
    else if (fl & kFlagRankOverflow) s = fail(ctx, HMLE_ERR_RANK_OVERFLOW, "ACA did not converge within its capacity");
  }
  if (s == HMLE_OK) {
    double mr;
    s = rank_stats(ctx, t, h->rank_c, &h->max_rank_c, &mr);
  }
  if (s != HMLE_OK) { free_hm(ctx->st, h); delete h; return s; }
  *out = h;
  return HMLE_OK;
}

void hmle_hmatrix_destroy(hmle_hmatrix *h) {
  if (!h) return;
  cudaStream_t st = nullptr;
  cudaDeviceSynchronize();
  free_hm(st, h);
  cudaStreamSynchronize(st);
  delete h;
}

hmle_status hmle_hmatrix_matvec(hmle_ctx *ctx, const hmle_hmatrix *h, const double *x, double *y) {
  if (!ctx || !h || !x || !y) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  const hmle_tree *t = h->tree;
  const Plan &P = t->plan;
  cudaStream_t st = ctx->st;
  const int64_t n = t->n;
  const int nlr = (int)t->lr_ids.size();
  double *xd = nullptr, *xp = nullptr, *yp = nullptr, *tb = nullptr, *yo = nullptr;
  bool owned = false;
  hmle_status s = stage_vec(ctx, x, n, &xd, &owned);
  if (s != HMLE_OK) return s;
  CK(cudaMallocAsync(&xp, sizeof(double) * n, st), "alloc");
  CK(cudaMallocAsync(&yp, sizeof(double) * n, st), "alloc");
  CK(cudaMallocAsync(&yo, sizeof(double) * n, st), "alloc");
  CK(cudaMallocAsync(&tb, sizeof(double) * std::max(nlr, 1) * 2 * P.kc, st), "alloc");
  launch_permute_in(st, xd, t->T.perm, n, xp);
  AsmArgs A{};
  A.blocks = t->dp.blocks; A.lr_ids = t->dp.lr_ids; A.xyz = t->T.xyz; A.n = n; A.d = t->d;
  A.tab = h->tab; A.inv_ell = 1.0 / h->th.ell; A.sigma2 = h->th.sigma2; A.tau2 = h->th.tau2;
  A.kc = P.kc; A.uc = h->uc; A.rank_c = h->rank_c; A.cnorm = h->cnorm; A.flags = h->flags;
  A.thd = h->thd; A.Cd = h->Cd; A.b = P.b;
  CmvLists L{P.nleaf, t->dp.leaf_beg, t->dp.mv_row0, t->dp.mv_blocks, t->dp.mvt_row0,
             t->dp.mvt_blocks, t->dp.lr_slot};
  launch_cmatvec(st, A, nlr, L, xp, tb, yp);
  launch_permute_out(st, yp, t->T.perm, n, yo);       // y[perm[k]] = yp[k]
  CK(cudaGetLastError(), "matvec launch");
  CK(cudaMemcpyAsync(y, yo, sizeof(double) * n, cudaMemcpyDefault, st), "copy");
  CK(cudaStreamSynchronize(st), "sync");
  if (owned) cudaFreeAsync(xd, st);
  cudaFreeAsync(xp, st);
  cudaFreeAsync(yp, st);
  cudaFreeAsync(yo, st);
  cudaFreeAsync(tb, st);
  CK(cudaStreamSynchronize(st), "sync");
  return HMLE_OK;
}

hmle_status hmle_factor(hmle_ctx *ctx, const hmle_hmatrix *h, const double *Z, hmle_hfactor **out) {
  if (!ctx || !h || !out) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  const hmle_tree *t = h->tree;
  hmle_hfactor *f = new (std::nothrow) hmle_hfactor();
  if (!f) return HMLE_ERR_OOM;
  hmle_status s = alloc_f(ctx, t, f);
  double *zd = nullptr;
  bool owned = false;
  if (s == HMLE_OK && Z) s = stage_vec(ctx, Z, t->n, &zd, &owned);
  if (s == HMLE_OK) s = do_factor(ctx, t, h, zd, f);
  if (s == HMLE_OK && zd && is_mixed(t->opts.precision)) s = mixed_quad(ctx, t, h, f, zd);
  if (owned) cudaFreeAsync(zd, ctx->st);
  if (s == HMLE_OK) s = rank_stats(ctx, t, f->rank_l, &f->max_rank_l, &f->mean_rank_l);
  if (s != HMLE_OK) { free_f(ctx->st, f); delete f; return s; }
  *out = f;
  return HMLE_OK;
}

void hmle_factor_destroy(hmle_hfactor *f) {
  if (!f) return;
  cudaStream_t st = nullptr;
  cudaDeviceSynchronize();
  free_f(st, f);
  cudaStreamSynchronize(st);
  delete f;
}

hmle_status hmle_loglik(hmle_ctx *ctx, const hmle_hfactor *fc, const double *Z, double *ll,
                        double *logdet, double *quad) {
  if (!ctx || !fc || !ll) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  hmle_hfactor *f = const_cast<hmle_hfactor *>(fc);
  const hmle_tree *t = f->h->tree;
  const double n = (double)t->n;
  if (Z) {
    // forward solve of this Z through the stored factor: w = L^{-1} P Z
    cudaStream_t st = ctx->st;
    const Plan &P = t->plan;
    double *zd = nullptr;
    bool owned = false;
    hmle_status s = stage_vec(ctx, Z, t->n, &zd, &owned);
    if (s != HMLE_OK) return s;
    const PanelDesc &rp = P.panels[P.rhs_panel];
    launch_permute_in(st, zd, t->T.perm, t->n, f->W + rp.off);
    FactorArgs F = make_fargs(t, f->h, f);
    F.hts = t->dp.hts_rhs;
    F.urows = t->dp.urows_rhs;
    F.uents = t->dp.uents_rhs;
    launch_solve(st, F, P, t->dp.wpan_rhs);
    launch_finalize(st, f->ldp, P.nleaf, f->W + rp.off, t->n, f->out);
    double out[2];
    CK(cudaGetLastError(), "solve launch");
    CK(cudaMemcpyAsync(out, f->out, sizeof(out), cudaMemcpyDeviceToHost, st), "result copy");
    CK(cudaStreamSynchronize(st), "solve sync");
    if (owned) cudaFreeAsync(zd, st);
    f->quad = out[1];
    f->has_rhs = true;
  } else if (!f->has_rhs) {
    return fail(ctx, HMLE_ERR_INVALID_ARG, "no Z: the factor was built without a right-hand side");
  }
  *ll = -0.5 * n * std::log(2.0 * M_PI) - 0.5 * f->logdet - 0.5 * f->quad;
  if (logdet) *logdet = f->logdet;
  if (quad) *quad = f->quad;
  return HMLE_OK;
}

}  // extern "C"

namespace {

// x = C~^{-1} P Z in cluster order, left in the factor's right-hand-side
// panel (forward sweep, q, backward sweep); *xout = that panel.  zd: Z in
// the caller's order, on the device.
hmle_status solve_cluster(hmle_ctx *ctx, hmle_hfactor *f, const double *zd, double **xout) {
  const hmle_tree *t = f->h->tree;
  const Plan &P = t->plan;
  cudaStream_t st = ctx->st;
  double *hb = nullptr;
  int maxh = 1;
  for (int K = 0; K < P.nleaf; ++K) maxh = std::max(maxh, P.bh0[K + 1] - P.bh0[K]);
  unsigned *bar = nullptr;
  CK(cudaMallocAsync(&hb, sizeof(double) * (size_t)maxh * P.kcap, st), "alloc");
  CK(cudaMallocAsync(&bar, 4 * sizeof(unsigned), st), "alloc");
  CK(cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st), "memset");
  const PanelDesc &rp = P.panels[P.rhs_panel];
  double *w = f->W + rp.off;
  launch_permute_in(st, zd, t->T.perm, t->n, w);
  FactorArgs F = make_fargs(t, f->h, f);
  F.hts = t->dp.hts_rhs;
  F.urows = t->dp.urows_rhs;
  F.uents = t->dp.uents_rhs;
  if (t->coop) {   // one cooperative launch per sweep
    CK(persistent_solve(st, F, t->sp, w, F.ws, bar, false), "forward sweep");   // w = L^{-1} P Z
    launch_finalize(st, f->ldp, P.nleaf, w, t->n, f->out);
    CK(persistent_solve(st, F, t->sp, w, hb, bar, true), "backward sweep");     // v = L^{-T} w
  } else {
    launch_solve(st, F, P, t->dp.wpan_rhs);
    launch_finalize(st, f->ldp, P.nleaf, w, t->n, f->out);
    launch_backward(st, F, P, w, t->dp.bh_blocks, t->dp.bupd, t->dp.bents, hb);
  }
  double out[2];
  unsigned berr = 0;
  CK(cudaGetLastError(), "solve launch");
  CK(cudaMemcpyAsync(out, f->out, sizeof(out), cudaMemcpyDeviceToHost, st), "copy");
  CK(cudaMemcpyAsync(&berr, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st), "copy");
  CK(cudaStreamSynchronize(st), "sync");
  cudaFreeAsync(bar, st);
  cudaFreeAsync(hb, st);
  if (berr) return fail(ctx, HMLE_ERR_TIMEOUT, "solve: a barrier wait of the persistent sweep ran out");
  f->quad = out[1];                   // the quadratic form now belongs to this Z
  f->has_rhs = true;
  *xout = w;
  return HMLE_OK;
}

}  // namespace

extern "C" {

hmle_status hmle_solve(hmle_ctx *ctx, const hmle_hfactor *fc, const double *Z, double *X) {
  if (!ctx || !fc || !Z || !X) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  hmle_hfactor *f = const_cast<hmle_hfactor *>(fc);
  const hmle_tree *t = f->h->tree;
  cudaStream_t st = ctx->st;
  double *zd = nullptr, *xo = nullptr, *w = nullptr;
  bool owned = false;
  hmle_status s = stage_vec(ctx, Z, t->n, &zd, &owned);
  if (s != HMLE_OK) return s;
  CK(cudaMallocAsync(&xo, sizeof(double) * t->n, st), "alloc");
  s = solve_cluster(ctx, f, zd, &w);
  if (s == HMLE_OK) {
    launch_permute_out(st, w, t->T.perm, t->n, xo);
    CK(cudaGetLastError(), "permute launch");
    CK(cudaMemcpyAsync(X, xo, sizeof(double) * t->n, cudaMemcpyDefault, st), "copy");
  }
  if (owned) cudaFreeAsync(zd, st);
  cudaFreeAsync(xo, st);
  CK(cudaStreamSynchronize(st), "sync");
  return s;
}

hmle_status hmle_predict(hmle_ctx *ctx, const hmle_hfactor *fc, const double *Z1,
                         const double *locs2, int64_t m, double *Z2) {
  if (!ctx || !fc || !Z1 || !locs2 || !Z2 || m < 1) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  hmle_hfactor *f = const_cast<hmle_hfactor *>(fc);
  const hmle_tree *t = f->h->tree;
  const hmle_hmatrix *h = f->h;
  cudaStream_t st = ctx->st;
  double *zd = nullptr, *l2 = nullptr, *w = nullptr, *out = nullptr;
  bool zown = false, lown = false;
  hmle_status s = stage_vec(ctx, Z1, t->n, &zd, &zown);
  if (s != HMLE_OK) return s;
  s = stage_vec(ctx, locs2, m * t->d, &l2, &lown);
  if (s != HMLE_OK) { if (zown) cudaFreeAsync(zd, st); return s; }
  CK(cudaMallocAsync(&out, sizeof(double) * m, st), "alloc");
  s = solve_cluster(ctx, f, zd, &w);                 // w = C~^{-1} Z1, cluster order
  if (s == HMLE_OK) {
    // Z2 = C21 w, C21 generated from the table at the factor's theta
    launch_cross_matvec(st, h->tab, t->T.xyz, t->n, t->d, l2, m, 1.0 / h->th.ell, h->th.sigma2, w, out);
    CK(cudaGetLastError(), "cross matvec launch");
    CK(cudaMemcpyAsync(Z2, out, sizeof(double) * m, cudaMemcpyDefault, st), "copy");
  }
  if (zown) cudaFreeAsync(zd, st);
  if (lown) cudaFreeAsync(l2, st);
  cudaFreeAsync(out, st);
  CK(cudaStreamSynchronize(st), "sync");
  return s;
}

hmle_status hmle_loglik_eval(hmle_ctx *ctx, const hmle_tree *tc, const hmle_theta *th,
                             const double *Z, double *ll, hmle_eval_info *info) {
  if (!ctx || !tc || !Z || !ll) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!theta_ok(th)) return fail(ctx, HMLE_ERR_INVALID_ARG, "theta out of range");
  hmle_tree *t = const_cast<hmle_tree *>(tc);
  hmle_status s = HMLE_OK;
  if (!t->work) {
    t->work = new (std::nothrow) Work();
    if (!t->work) return HMLE_ERR_OOM;
    s = alloc_hm(ctx, t, &t->work->H);
    if (s == HMLE_OK) s = alloc_f(ctx, t, &t->work->F);
    if (s == HMLE_OK) {
      cudaError_t e = cudaMallocAsync(&t->work->zdev, sizeof(double) * t->n, ctx->st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "alloc z");
    }
    if (s != HMLE_OK) {
      free_hm(ctx->st, &t->work->H);
      free_f(ctx->st, &t->work->F);
      delete t->work;
      t->work = nullptr;
      return s;
    }
  }
  Work &w = *t->work;
  const double *zd = Z;
  if (!is_device_ptr(Z)) {
    CK(cudaMemcpyAsync(w.zdev, Z, sizeof(double) * t->n, cudaMemcpyHostToDevice, ctx->st), "copy z");
    zd = w.zdev;
  }
  s = do_assemble(ctx, t, th, &w.H);
  if (s == HMLE_OK) s = do_factor(ctx, t, &w.H, zd, &w.F, t->graphs ? &w : nullptr);
  if (s == HMLE_OK && is_mixed(t->opts.precision)) s = mixed_quad(ctx, t, &w.H, &w.F, zd);
  const double n = (double)t->n;
  double L = -0.5 * n * std::log(2.0 * M_PI) - 0.5 * w.F.logdet - 0.5 * w.F.quad;
  *ll = (s == HMLE_OK) ? L : -INFINITY;
  if (info) {
    info->logdet = w.F.logdet;
    info->quad = w.F.quad;
    info->loglik = *ll;
    info->status = s;
    info->kernel_launches = w.F.launches;
    info->pcg_iters = w.F.pcg_iters;
    info->pcg_relres = w.F.pcg_relres;
    info->flops = 0.0;
    if (s == HMLE_OK) {   // algorithmic flops of the sweep, from the plan and this evaluation's ranks
      const Plan &P = t->plan;
      std::vector<int32_t> rc(P.blocks.size()), rl(P.blocks.size()), kp(std::max<size_t>(P.lrt.size(), 1));
      double jf = 0.0;
      cudaStream_t st = ctx->st;
      cudaError_t e = cudaMemcpyAsync(rc.data(), w.H.rank_c, sizeof(int32_t) * rc.size(), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(rl.data(), w.F.rank_l, sizeof(int32_t) * rl.size(), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(kp.data(), w.F.kept, sizeof(int32_t) * kp.size(), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaMemcpyAsync(&jf, ctx->d_jacobi, sizeof(double), cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
      if (e == cudaSuccess)
        for (int k = 0; k < KK_COUNT; ++k)
          info->flops += tally_flops(P, k, rc, rl, kp, t->opts.oversample, jf);
      else
        cudaGetLastError();
    }
    double mr = 0;
    int mx = 0;
    if (rank_stats(ctx, t, w.H.rank_c, &mx, &mr) == HMLE_OK) info->max_rank_c = mx;
    if (rank_stats(ctx, t, w.F.rank_l, &mx, &mr) == HMLE_OK) {
      info->max_rank_l = mx;
      info->mean_rank_l = mr;
    }
  }
  return s;
}

namespace {

// Grow a tree's pool of evaluation buffers (each with its own stream pair)
// to at least W.
hmle_status ensure_pool(hmle_ctx *ctx, hmle_tree *t, int W) {
  while ((int)t->pool.size() < W) {
    Work *w = new (std::nothrow) Work();
    if (!w) return HMLE_ERR_OOM;
    cudaError_t e = cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&w->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaMalloc(&w->d_jacobi, sizeof(double));
    if (e != cudaSuccess) { free_work(w); return cuda_fail(ctx, e, "batch streams"); }
    hmle_ctx wc;                       // a context view on the work's streams
    wc.st = w->st; wc.side = w->side; wc.ev_fork = w->ev_fork; wc.ev_join = w->ev_join;
    wc.d_jacobi = w->d_jacobi;
    hmle_status s = alloc_hm(&wc, t, &w->H);
    if (s == HMLE_OK) s = alloc_f(&wc, t, &w->F);
    if (s == HMLE_OK) {
      e = cudaMallocAsync(&w->zdev, sizeof(double) * t->n, w->st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(w->st);
      if (e != cudaSuccess) s = cuda_fail(ctx, e, "batch alloc");
    }
    wc.d_jacobi = nullptr;
    if (s != HMLE_OK) { free_work(w); return fail(ctx, s, wc.err.empty() ? ctx->err : wc.err); }
    t->pool.push_back(w);
  }
  return HMLE_OK;
}

// The batch of nz evaluations of tree t (created on first use, kept with the
// tree): one allocation for all nz buffer sets, at a stride of the size of
// one set, and per-evaluation views of it.
hmle_status ensure_group(hmle_ctx *ctx, hmle_tree *t, int nz, int sub, Group **out) {
  for (Group *g : t->groups)
    if (g->nz == nz && g->sub == sub) { *out = g; return HMLE_OK; }
  // one batch per tree: a batch of another size is released first (its
  // streams are idle: every call waits for its batch before returning)
  for (Group *g : t->groups) free_group(g);
  t->groups.clear();
  const Plan &P = t->plan;
  const int64_t nb = std::max<int64_t>((int64_t)P.blocks.size(), 1);
  int64_t off = 0;
  auto take = [&](int64_t bytes) { const int64_t o = off; off += (std::max<int64_t>(bytes, 8) + 255) & ~(int64_t)255; return o; };
  const int64_t o_tab = take(8 * (int64_t)kTableWords), o_uc = take(8 * P.uc_words), o_cd = take(8 * P.dense_words);
  const int64_t o_rc = take(4 * nb), o_cn = take(8 * nb), o_th = take(sizeof(ThetaDev)), o_hf = take(4);
  const int64_t o_d = take(8 * P.dense_words), o_u = take(8 * P.u_words), o_w = take(8 * P.w_words);
  const int64_t o_ws = take(8 * P.ws_max), o_rl = take(4 * nb), o_kp = take(4 * std::max<int64_t>((int64_t)P.lrt.size(), 1));
  const int64_t o_ld = take(8 * (int64_t)P.nleaf), o_ff = take(4), o_out = take(16), o_jac = take(8);
  // the mixed forms' PCG workspace (right-hand side + vectors), as mixed_prepare sizes it
  int64_t o_pcg = -1;
  if (is_mixed(t->opts.precision)) {
    int hmax = 1;
    for (int K = 0; K < P.nleaf; ++K) hmax = std::max(hmax, P.bh0[K + 1] - P.bh0[K]);
    o_pcg = take(8 * (t->n + pcg_words(t->n, (int)t->lr_ids.size(), P.kc, hmax * P.kcap) + 2));
  }
  Group *g = new (std::nothrow) Group();
  if (!g) return fail(ctx, HMLE_ERR_OOM, "batch");
  g->nz = nz;
  g->sub = std::max(1, std::min(sub, nz));
  g->stride = off;
  const int ns = g->nsub();
  g->st.assign(ns, nullptr); g->side.assign(ns, nullptr);
  g->ev_fork.assign(ns, nullptr); g->ev_join.assign(ns, nullptr); g->done.assign(ns, nullptr);
  g->exec.assign(ns, nullptr); g->launches.assign(ns, 0);
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < ns && e == cudaSuccess; ++k) {
    e = cudaStreamCreateWithFlags(&g->st[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&g->side[k], cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_fork[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->ev_join[k], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&g->done[k], cudaEventDisableTiming);
  }
  if (e == cudaSuccess) e = cudaMalloc(&g->arena, (size_t)(off * nz));
  if (e == cudaSuccess) e = cudaMemset(g->arena, 0, (size_t)(off * nz));
  if (e == cudaSuccess) e = cudaMalloc(&g->bar, 3 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemset(g->bar, 0, 3 * sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMallocHost(&g->host, sizeof(double) * (4 + 4 * (size_t)nz));
  if (e != cudaSuccess) { free_group(g); return cuda_fail(ctx, e, "batch buffers"); }
  for (int z = 0; z < nz; ++z) {
    Work *w = new (std::nothrow) Work();
    if (!w) { free_group(g); return fail(ctx, HMLE_ERR_OOM, "batch"); }
    g->w.push_back(w);
    e = cudaStreamCreateWithFlags(&w->st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&w->done, cudaEventDisableTiming);
    if (e != cudaSuccess) { free_group(g); return cuda_fail(ctx, e, "batch streams"); }
    char *b = g->arena + (int64_t)z * off;
    w->H.tree = t;
    w->H.tab = (double *)(b + o_tab); w->H.uc = (double *)(b + o_uc); w->H.Cd = (double *)(b + o_cd);
    w->H.rank_c = (int32_t *)(b + o_rc); w->H.cnorm = (double *)(b + o_cn);
    w->H.thd = (ThetaDev *)(b + o_th); w->H.flags = (int *)(b + o_hf);
    w->F.D = (double *)(b + o_d); w->F.U = (double *)(b + o_u); w->F.W = (double *)(b + o_w);
    w->F.ws = (double *)(b + o_ws); w->F.rank_l = (int32_t *)(b + o_rl); w->F.kept = (int32_t *)(b + o_kp);
    w->F.ldp = (double *)(b + o_ld); w->F.flags = (int *)(b + o_ff); w->F.out = (double *)(b + o_out);
    w->d_jacobi = (double *)(b + o_jac);
    if (o_pcg >= 0) w->F.pcg = (double *)(b + o_pcg);
  }
  t->groups.push_back(g);
  *out = g;
  return HMLE_OK;
}

// The sweep of the cnt evaluations z0 .. z0 + cnt - 1 of a batch (one
// sub-batch): per-evaluation state reset (flags, ranks, Jacobi counters, by
// strided memsets), the steps with gridDim.z = cnt, and the per-evaluation
// log-det / quadratic-form reductions.  Returns the number of launches.
int64_t launch_group_sweep(hmle_ctx *gc, const hmle_tree *t, Group *g, int z0, int cnt, Prof *prof) {
  cudaStream_t st = gc->st;
  const Plan &P = t->plan;
  Work *w0 = g->w[z0];
  FactorArgs F = make_fargs(t, &w0->H, &w0->F);
  F.jacobi_flops = w0->d_jacobi;
  F.nz = cnt;
  F.zstride = g->stride;
  const size_t nb = std::max<size_t>(P.blocks.size(), 1);
  cudaMemset2DAsync(F.flags, (size_t)g->stride, 0, sizeof(int), cnt, st);
  cudaMemset2DAsync(F.rank_l, (size_t)g->stride, 0, sizeof(int32_t) * nb, cnt, st);
  cudaMemset2DAsync(w0->d_jacobi, (size_t)g->stride, 0, sizeof(double), cnt, st);
  int64_t nk = 0;
  for (int K = 0; K < P.nleaf; ++K)
    nk += launch_step(st, gc->side, gc->ev_fork, gc->ev_join, F, P.steps[K], K, P, prof);
  const PanelDesc &rp = P.panels[P.rhs_panel];
  for (int z = z0; z < z0 + cnt; ++z)
    launch_finalize(st, g->w[z]->F.ldp, P.nleaf, g->w[z]->F.W + rp.off, t->n, g->w[z]->F.out);
  return nk + cnt;
}

// m evaluations of tree t at thetas (Z on the device), in waves of up to nz:
// a wave runs as sub-batches of `sub` evaluations, each with one launch per
// kernel for the whole sub-batch, side by side on their own streams (the
// last wave is filled with copies of its last theta, whose results are not
// reported).  The mixed forms then solve every evaluation of the wave with
// one PCG in lockstep.
hmle_status run_group(hmle_ctx *ctx, hmle_tree *t, const hmle_theta *thetas, int m, const double *zd,
                      int nz, int sub, cudaEvent_t zready, double *ll, int32_t *status, double *ld_out,
                      double *q_out) {
  Group *g = nullptr;
  hmle_status s0 = ensure_group(ctx, t, nz, sub, &g);
  if (s0 != HMLE_OK) return s0;
  const Plan &P = t->plan;
  const PanelDesc &rp = P.panels[P.rhs_panel];
  const int ns = g->nsub();
  auto view = [&](int k) {   // a context view on sub-batch k's streams
    hmle_ctx c;
    c.st = g->st[k]; c.side = g->side[k]; c.ev_fork = g->ev_fork[k]; c.ev_join = g->ev_join[k];
    c.d_jacobi = g->w[k * g->sub]->d_jacobi;
    return c;
  };
  Prof *prof = ctx->prof.kind >= 0 ? &ctx->prof : nullptr;
  hmle_status first = HMLE_OK;
  for (int k = 0; k < ns; ++k) CK(cudaStreamWaitEvent(g->st[k], zready, 0), "stream wait");
  for (int i0 = 0; i0 < m; i0 += nz) {
    const int cnt = std::min(nz, m - i0);
    std::vector<hmle_status> fs(nz, HMLE_OK);
    std::vector<std::string> errs(nz);
    int nev = 0;
    for (int k = 0; k < ns; ++k) {
      const int z0 = k * g->sub, zc = std::min(g->sub, nz - z0);
      hmle_ctx gc = view(k);
      for (int z = z0; z < z0 + zc; ++z) {
        Work *w = g->w[z];
        const hmle_theta *th = &thetas[i0 + std::min(z, cnt - 1)];
        fs[z] = do_assemble(&gc, t, th, &w->H);
        launch_permute_in(g->st[k], zd, t->T.perm, t->n, w->F.W + rp.off);
        w->F.h = &w->H;
        w->F.has_rhs = true;
        if (fs[z] != HMLE_OK) errs[z] = gc.err;
      }
      if (prof || !t->graphs) {   // direct launches (CUDA events cannot be read inside a graph)
        if (prof) prof->used = nev;
        g->launches[k] = launch_group_sweep(&gc, t, g, z0, zc, prof);
        nev = prof ? prof->used : 0;
      } else {
        if (!g->exec[k]) {
          cudaGraph_t gr = nullptr;
          CK(cudaStreamBeginCapture(g->st[k], cudaStreamCaptureModeThreadLocal), "begin capture");
          const int64_t nk = launch_group_sweep(&gc, t, g, z0, zc, nullptr);
          cudaError_t e = cudaStreamEndCapture(g->st[k], &gr);
          if (e != cudaSuccess) return cuda_fail(ctx, e, "end capture");
          e = cudaGraphInstantiate(&g->exec[k], gr, 0);
          cudaGraphDestroy(gr);
          if (e != cudaSuccess) { g->exec[k] = nullptr; return cuda_fail(ctx, e, "graph instantiate"); }
          g->launches[k] = nk;
        }
        CK(cudaGraphLaunch(g->exec[k], g->st[k]), "graph launch");
      }
      CK(cudaEventRecord(g->done[k], g->st[k]), "event record");
    }
    CK(cudaGetLastError(), "batch launch");
    for (int k = 0; k < ns; ++k) CK(cudaStreamSynchronize(g->st[k]), "batch sync");
    if (prof) {
      prof_collect(prof, nev);
      for (int z = 0; z < cnt; ++z) {
        Work *w = g->w[z];
        std::vector<int32_t> rc(P.blocks.size()), rl(P.blocks.size()), kp(std::max<size_t>(P.lrt.size(), 1));
        double jf = 0.0;
        CK(cudaMemcpy(rc.data(), w->H.rank_c, sizeof(int32_t) * rc.size(), cudaMemcpyDeviceToHost), "ranks");
        CK(cudaMemcpy(rl.data(), w->F.rank_l, sizeof(int32_t) * rl.size(), cudaMemcpyDeviceToHost), "ranks");
        CK(cudaMemcpy(kp.data(), w->F.kept, sizeof(int32_t) * kp.size(), cudaMemcpyDeviceToHost), "kept");
        CK(cudaMemcpy(&jf, w->d_jacobi, sizeof(double), cudaMemcpyDeviceToHost), "jacobi");
        prof->flops += tally_flops(P, prof->kind, rc, rl, kp, t->opts.oversample, jf);
      }
    }
    // results; the mixed forms then solve for every evaluation of the wave
    // at once (one PCG in lockstep), or, without cooperative launches, run
    // their PCG solves interleaved on their own streams
    std::vector<PcgRun> runs(cnt);
    std::vector<int> live;
    const bool lockstep = is_mixed(t->opts.precision) && t->coop;
    for (int z = 0; z < cnt; ++z) {
      Work *w = g->w[z];
      w->F.launches = g->launches[z / g->sub] + kAssemblyLaunches + 1;
      hmle_ctx wc;
      wc.st = g->st[z / g->sub];
      if (fs[z] == HMLE_OK) fs[z] = finish_factor(&wc, t, &w->H, &w->F);
      if (fs[z] != HMLE_OK && errs[z].empty()) errs[z] = wc.err;
    }
    if (lockstep) {
      PcgRun R;
      hmle_ctx gc = view(0);
      hmle_status sp = mixed_prepare(&gc, t, &g->w[0]->H, &g->w[0]->F, zd, R);
      if (sp == HMLE_OK) {
        for (int z = 1; z < nz; ++z) launch_permute_in(g->st[0], zd, t->T.perm, t->n, g->w[z]->F.pcg);
        R.nz = nz;
        R.zs = g->stride / (int64_t)sizeof(double);
        R.Fs.nz = nz;
        R.Fs.zstride = g->stride;
        R.A.zstride = g->stride;
        R.bar = g->bar;
        R.host = g->host;
        R.hostz = g->host + 4;
        R.g_init = R.g_iter = nullptr;
        cudaError_t e = cudaMemsetAsync(g->bar, 0, 3 * sizeof(unsigned), g->st[0]);
        if (e == cudaSuccess) e = pcg_batch_start(R);
        bool fin = false;
        while (e == cudaSuccess && !fin) {
          e = cudaStreamSynchronize(g->st[0]);
          if (e == cudaSuccess) e = pcg_batch_poll(R, &fin);
        }
        if (e != cudaSuccess) sp = cuda_fail(&gc, e, "pcg");
      }
      for (int z = 0; z < cnt; ++z) {
        if (fs[z] != HMLE_OK) continue;
        hmle_hfactor &F = g->w[z]->F;
        if (sp != HMLE_OK) { fs[z] = sp; errs[z] = gc.err; continue; }
        if (R.timed_out) {
          fs[z] = HMLE_ERR_TIMEOUT;
          errs[z] = "PCG: a barrier wait of the persistent sweep ran out";
          continue;
        }
        F.quad = R.qz[z];
        F.pcg_iters = R.itz[z];
        F.pcg_relres = R.relz[z];
        F.has_rhs = true;
        if (!(F.pcg_relres <= t->opts.pcg_tol) || !std::isfinite(F.quad)) {
          fs[z] = HMLE_ERR_NOT_CONVERGED;
          errs[z] = "PCG: relative residual above pcg_tol after pcg_max_iter";
        }
      }
    }
    for (int z = 0; z < cnt && !lockstep; ++z) {
      Work *w = g->w[z];
      hmle_ctx wc;
      if (fs[z] == HMLE_OK && is_mixed(t->opts.precision)) {
        wc.st = w->st;
        cudaStreamWaitEvent(w->st, g->done[z / g->sub], 0);
        fs[z] = mixed_prepare(&wc, t, &w->H, &w->F, zd, runs[z]);
        if (fs[z] == HMLE_OK) {
          cudaError_t e = pcg_start(runs[z]);
          if (e != cudaSuccess) fs[z] = cuda_fail(&wc, e, "pcg");
          else live.push_back(z);
        }
      }
      if (fs[z] != HMLE_OK && errs[z].empty()) errs[z] = wc.err;
    }
    while (!live.empty()) {
      std::vector<int> next;
      for (int z : live) {
        bool fin = false;
        hmle_ctx wc;
        cudaError_t e = cudaStreamSynchronize(runs[z].st);
        if (e == cudaSuccess) e = pcg_poll(runs[z], &fin);
        if (e != cudaSuccess) {
          fs[z] = cuda_fail(&wc, e, "pcg");
          errs[z] = wc.err;
        } else if (fin) {
          fs[z] = mixed_result(&wc, t, &g->w[z]->F, runs[z]);
          if (fs[z] != HMLE_OK) errs[z] = wc.err;
        } else {
          next.push_back(z);
        }
      }
      live.swap(next);
    }
    for (int z = 0; z < cnt; ++z) {
      const int i = i0 + z;
      const hmle_hfactor &F = g->w[z]->F;
      const hmle_status s = fs[z];
      const double nn = (double)t->n;
      ll[i] = (s == HMLE_OK) ? -0.5 * nn * std::log(2.0 * M_PI) - 0.5 * F.logdet - 0.5 * F.quad : -INFINITY;
      if (ld_out) ld_out[i] = (s == HMLE_OK) ? F.logdet : NAN;
      if (q_out) q_out[i] = (s == HMLE_OK) ? F.quad : NAN;
      if (status) status[i] = s;
      if (!per_eval_status(s) && first == HMLE_OK) {
        first = s;
        ctx->err = errs[z];
      }
    }
  }
  return first;
}

// One evaluation request of a batch: tree, theta, and Z already on the device.
struct TaskRef {
  hmle_tree *t;
  const hmle_theta *th;
  const double *zd;
};

// a15: evaluate the tasks in waves of W; inside a wave every task runs on a
// buffer of its tree's pool, on its own streams (replaying the tree's
// captured sweep), and the wave is collected in task order.  zready: an
// event after which every Z is readable.
hmle_status run_waves(hmle_ctx *ctx, const std::vector<TaskRef> &tasks, int W, cudaEvent_t zready,
                      double *ll, int32_t *status, double *ld_out = nullptr, double *q_out = nullptr) {
  const int m = (int)tasks.size();
  hmle_status first = HMLE_OK;
  // the last task of every tree: once its wave is collected, the tree's
  // evaluation buffers are released, so that many trees of uneven n can be
  // evaluated in one call without holding every tree's buffers at once
  std::vector<std::pair<hmle_tree *, int>> last;
  for (int i = 0; i < m; ++i) {
    bool found = false;
    for (auto &u : last)
      if (u.first == tasks[i].t) { u.second = i; found = true; }
    if (!found) last.push_back({tasks[i].t, i});
  }
  for (int i0 = 0; i0 < m; i0 += W) {
    const int cnt = std::min(W, m - i0);
    std::vector<Work *> ws(cnt, nullptr);
    {
      std::vector<std::pair<hmle_tree *, int>> used;   // pool slots taken per tree
      for (int k = 0; k < cnt; ++k) {
        hmle_tree *t = tasks[i0 + k].t;
        int slot = 0;
        for (auto &u : used)
          if (u.first == t) slot = ++u.second;
        if (slot == 0) used.push_back({t, 0});
        hmle_status s = ensure_pool(ctx, t, slot + 1);
        if (s != HMLE_OK) return s;
        ws[k] = t->pool[slot];
      }
    }
    // launch every evaluation of the wave asynchronously
    for (int k = 0; k < cnt; ++k) {
      const TaskRef &T = tasks[i0 + k];
      Work *w = ws[k];
      hmle_ctx wc;
      wc.st = w->st; wc.side = w->side; wc.ev_fork = w->ev_fork; wc.ev_join = w->ev_join;
      wc.d_jacobi = w->d_jacobi;
      CK(cudaStreamWaitEvent(w->st, zready, 0), "stream wait");
      hmle_status s = do_assemble(&wc, T.t, T.th, &w->H);
      if (s == HMLE_OK) s = launch_factor_async(&wc, T.t, &w->H, T.zd, &w->F, T.t->graphs ? w : nullptr);
      wc.d_jacobi = nullptr;
      if (s != HMLE_OK) { if (status) status[i0 + k] = s; if (first == HMLE_OK) { first = s; ctx->err = wc.err; } }
      else if (status) status[i0 + k] = HMLE_OK;
    }
    // collect the factorisations; mixed-form evaluations then run their PCG
    // solves interleaved across the wave's streams
    std::vector<hmle_status> fs(cnt, HMLE_OK);
    std::vector<PcgRun> runs(cnt);
    std::vector<int> live;
    std::vector<std::string> errs(cnt);
    for (int k = 0; k < cnt; ++k) {
      const TaskRef &T = tasks[i0 + k];
      Work *w = ws[k];
      hmle_ctx wc;
      wc.st = w->st; wc.side = w->side;
      fs[k] = finish_factor(&wc, T.t, &w->H, &w->F);
      if (fs[k] == HMLE_OK && is_mixed(T.t->opts.precision)) {
        fs[k] = mixed_prepare(&wc, T.t, &w->H, &w->F, T.zd, runs[k]);
        if (fs[k] == HMLE_OK) {
          cudaError_t e = pcg_start(runs[k]);
          if (e != cudaSuccess) fs[k] = cuda_fail(&wc, e, "pcg");
          else live.push_back(k);
        }
      }
      errs[k] = wc.err;
    }
    while (!live.empty()) {
      std::vector<int> next;
      for (int k : live) {
        bool fin = false;
        cudaError_t e = cudaStreamSynchronize(runs[k].st);
        if (e == cudaSuccess) e = pcg_poll(runs[k], &fin);
        if (e != cudaSuccess) {
          hmle_ctx wc;
          fs[k] = cuda_fail(&wc, e, "pcg");
          errs[k] = wc.err;
        } else if (fin) {
          hmle_ctx wc;
          fs[k] = mixed_result(&wc, tasks[i0 + k].t, &ws[k]->F, runs[k]);
          errs[k] = wc.err;
        } else {
          next.push_back(k);
        }
      }
      live.swap(next);
    }
    for (int k = 0; k < cnt; ++k) {
      const TaskRef &T = tasks[i0 + k];
      Work *w = ws[k];
      hmle_ctx wc;
      wc.err = errs[k];
      hmle_status s = fs[k];
      const int i = i0 + k;
      const double nn = (double)T.t->n;
      ll[i] = (s == HMLE_OK) ? -0.5 * nn * std::log(2.0 * M_PI) - 0.5 * w->F.logdet - 0.5 * w->F.quad
                             : -INFINITY;
      if (ld_out) ld_out[i] = (s == HMLE_OK) ? w->F.logdet : NAN;
      if (q_out) q_out[i] = (s == HMLE_OK) ? w->F.quad : NAN;
      if (status && status[i] == HMLE_OK) status[i] = s;
      if (!per_eval_status(s) && first == HMLE_OK) {
        first = s;
        ctx->err = wc.err;
      }
    }
    for (auto &u : last)   // trees with no task after this wave: release their buffers
      if (u.second >= i0 && u.second < i0 + cnt) {
        for (Work *w : u.first->pool) free_work(w);
        u.first->pool.clear();
      }
  }
  return first;
}

// m evaluations on one tree (Z on the device); ll, and optionally log|C~| and
// Z^T C~^{-1} Z, per evaluation.
hmle_status batch_eval(hmle_ctx *ctx, hmle_tree *t, const hmle_theta *thetas, int m,
                       const double *zd, int W, double *ll, int32_t *status, double *ld,
                       double *q) {
  cudaEvent_t zready;
  CK(cudaEventCreateWithFlags(&zready, cudaEventDisableTiming), "event");
  CK(cudaEventRecord(zready, ctx->st), "event record");
  hmle_status first = run_group(ctx, t, thetas, m, zd, std::min(W, std::max(m, 1)), t->opts.batch_size, zready,
                                ll, status, ld, q);
  cudaEventDestroy(zready);
  return first;
}

}  // namespace

hmle_status hmle_loglik_batch(hmle_ctx *ctx, const hmle_tree *tc, const hmle_theta *thetas,
                              int32_t m, const double *Z, int32_t concurrency, double *ll,
                              int32_t *status) {
  if (!ctx || !tc || !thetas || !Z || !ll || m < 0) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (concurrency <= 0) concurrency = 8;
  if (concurrency > 64) concurrency = 64;
  for (int i = 0; i < m; ++i)
    if (!theta_ok(&thetas[i])) return fail(ctx, HMLE_ERR_INVALID_ARG, "theta out of range");
  if (m == 0) return HMLE_OK;
  hmle_tree *t = const_cast<hmle_tree *>(tc);
  const int W = std::min<int>(concurrency, std::max(m, 1));
  // stage Z once (shared by every evaluation, read-only)
  double *zd = nullptr;
  bool owned = false;
  hmle_status s0 = stage_vec(ctx, Z, t->n, &zd, &owned);
  if (s0 != HMLE_OK) return s0;
  cudaEvent_t zready;
  CK(cudaEventCreateWithFlags(&zready, cudaEventDisableTiming), "event");
  CK(cudaEventRecord(zready, ctx->st), "event record");
  hmle_status first = run_group(ctx, t, thetas, m, zd, W, t->opts.batch_size, zready, ll, status, nullptr, nullptr);
  cudaEventDestroy(zready);
  if (owned) cudaFreeAsync(zd, ctx->st);
  cudaStreamSynchronize(ctx->st);
  return first;
}

}  // extern "C"

namespace {

// The retry ladder of a failed evaluation: the options of the next attempt
// after status s, or false when there is none.  A rank overflow first raises
// the rank capacity to its largest (56 columns plus 8 of oversampling; ACA
// of C then has 64), then loosens the accuracy tenfold per step up to 1e-3;
// a mixed-form evaluation whose PCG did not converge, or whose factor lost
// positive definiteness, is done again in FP64.
constexpr int kRetryRank = 56, kRetryOversample = 8;
constexpr double kRetryEpsMax = 1e-3;

bool next_attempt(hmle_opts &o, hmle_status s) {
  if (s == HMLE_ERR_NOT_CONVERGED || s == HMLE_ERR_NOT_SPD) {
    if (!is_mixed(o.precision)) return false;
    o.precision = HMLE_FP64;
    return true;
  }
  if (s != HMLE_ERR_RANK_OVERFLOW || o.fixed_rank > 0) return false;
  if (o.max_rank < kRetryRank) {
    o.max_rank = kRetryRank;
    o.oversample = kRetryOversample;
    return true;
  }
  if (o.aca_eps * 10.0 > kRetryEpsMax * (1.0 + 1e-12)) return false;
  o.aca_eps *= 10.0;
  return true;
}

bool same_opts(const hmle_opts &a, const hmle_opts &b) {
  return a.max_rank == b.max_rank && a.oversample == b.oversample && a.precision == b.precision &&
         a.aca_eps == b.aca_eps;
}

hmle_status multi_eval(hmle_ctx *ctx, const hmle_task *tasks, int32_t m, int32_t concurrency,
                       int32_t max_retries, double *ll, int32_t *status_out, hmle_retry_info *retry) {
  if (!ctx || !tasks || !ll || m < 0 || max_retries < 0) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (concurrency <= 0) concurrency = 8;
  if (concurrency > 64) concurrency = 64;
  for (int i = 0; i < m; ++i) {
    if (!tasks[i].tree || !tasks[i].Z) return fail(ctx, HMLE_ERR_INVALID_ARG, "null tree or Z in a task");
    if (!theta_ok(&tasks[i].theta)) return fail(ctx, HMLE_ERR_INVALID_ARG, "theta out of range");
  }
  if (m == 0) return HMLE_OK;
  const int W = std::min<int>(concurrency, std::max(m, 1));
  std::vector<int32_t> status(m, HMLE_OK);
  // stage every distinct Z once
  std::vector<const double *> src;
  std::vector<double *> dev;
  std::vector<bool> own;
  std::vector<TaskRef> refs(m);
  hmle_status s0 = HMLE_OK;
  for (int i = 0; i < m && s0 == HMLE_OK; ++i) {
    hmle_tree *t = const_cast<hmle_tree *>(tasks[i].tree);
    size_t q = 0;
    while (q < src.size() && src[q] != tasks[i].Z) ++q;
    if (q == src.size()) {
      double *zd = nullptr;
      bool owned = false;
      s0 = stage_vec(ctx, tasks[i].Z, t->n, &zd, &owned);
      src.push_back(tasks[i].Z);
      dev.push_back(zd);
      own.push_back(owned);
    }
    refs[i] = {t, &tasks[i].theta, dev[q]};
  }
  hmle_status first = s0;
  cudaEvent_t zready = nullptr;
  if (first == HMLE_OK) {
    if (cudaEventCreateWithFlags(&zready, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventRecord(zready, ctx->st) != cudaSuccess)
      first = fail(ctx, HMLE_ERR_CUDA, "event");
  }
  if (first == HMLE_OK) first = run_waves(ctx, refs, W, zready, ll, status.data());
  // retries: failed tasks again on trees derived from their own, one rung of
  // the ladder further per round, until they succeed or the ladder ends
  std::vector<hmle_opts> cur(m);
  std::vector<int32_t> tries(m, 0);
  for (int i = 0; i < m; ++i) cur[i] = tasks[i].tree->opts;
  struct Derived { const hmle_tree *src; hmle_opts o; hmle_tree *t; };
  std::vector<Derived> derived;
  for (int r = 0; r < max_retries && first == HMLE_OK; ++r) {
    std::vector<int> again;
    std::vector<TaskRef> rrefs;
    for (int i = 0; i < m && first == HMLE_OK; ++i) {
      if (status[i] == HMLE_OK) continue;
      hmle_opts o = cur[i];
      if (!next_attempt(o, (hmle_status)status[i])) continue;
      hmle_tree *dt = nullptr;
      for (const Derived &D : derived)
        if (D.src == tasks[i].tree && same_opts(D.o, o)) dt = D.t;
      if (!dt) {
        first = derive_tree(ctx, tasks[i].tree, o, &dt);
        if (first != HMLE_OK) break;
        derived.push_back({tasks[i].tree, o, dt});
      }
      cur[i] = o;
      ++tries[i];
      again.push_back(i);
      rrefs.push_back({dt, &tasks[i].theta, refs[i].zd});
    }
    if (again.empty() || first != HMLE_OK) break;
    std::vector<double> rll(again.size());
    std::vector<int32_t> rst(again.size(), HMLE_OK);
    first = run_waves(ctx, rrefs, std::min<int>(W, (int)again.size()), zready, rll.data(), rst.data());
    for (size_t k = 0; k < again.size(); ++k) {
      ll[again[k]] = rll[k];
      status[again[k]] = rst[k];
    }
  }
  if (zready) cudaEventDestroy(zready);
  for (const Derived &D : derived) hmle_tree_destroy(D.t);
  for (size_t q = 0; q < dev.size(); ++q)
    if (own[q] && dev[q]) cudaFreeAsync(dev[q], ctx->st);
  cudaStreamSynchronize(ctx->st);
  if (status_out) std::copy(status.begin(), status.end(), status_out);
  if (retry)
    for (int i = 0; i < m; ++i)
      retry[i] = hmle_retry_info{tries[i], cur[i].max_rank, cur[i].precision, cur[i].aca_eps};
  return first;
}

}  // namespace

extern "C" {

hmle_status hmle_loglik_multi(hmle_ctx *ctx, const hmle_task *tasks, int32_t m, int32_t concurrency,
                              double *ll, int32_t *status) {
  return multi_eval(ctx, tasks, m, concurrency, 0, ll, status, nullptr);
}

hmle_status hmle_loglik_multi_retry(hmle_ctx *ctx, const hmle_task *tasks, int32_t m, int32_t concurrency,
                                    int32_t max_retries, double *ll, int32_t *status,
                                    hmle_retry_info *retry) {
  if (max_retries > 8) return fail(ctx, HMLE_ERR_INVALID_ARG, "max_retries must be in [0, 8]");
  return multi_eval(ctx, tasks, m, concurrency, max_retries, ll, status, retry);
}

hmle_status hmle_simulate(hmle_ctx *ctx, const hmle_tree *tc, const hmle_theta *th,
                          const double *xi, double *Z) {
  if (!ctx || !tc || !xi || !Z) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!theta_ok(th)) return fail(ctx, HMLE_ERR_INVALID_ARG, "theta out of range");
  hmle_tree *t = const_cast<hmle_tree *>(tc);
  cudaStream_t st = ctx->st;
  const Plan &P = t->plan;
  const int64_t n = t->n;
  hmle_hmatrix *h = nullptr;
  hmle_status s = hmle_assemble(ctx, t, th, &h);
  if (s != HMLE_OK) return s;
  hmle_hfactor *f = new (std::nothrow) hmle_hfactor();
  if (!f) { hmle_hmatrix_destroy(h); return HMLE_ERR_OOM; }
  s = alloc_f(ctx, t, f);
  if (s == HMLE_OK) s = do_factor(ctx, t, h, nullptr, f);
  double *xd = nullptr, *xp = nullptr, *y = nullptr, *tw = nullptr, *zo = nullptr;
  bool owned = false;
  if (s == HMLE_OK) s = stage_vec(ctx, xi, n, &xd, &owned);
  if (s == HMLE_OK) {
    cudaError_t e = cudaMallocAsync(&xp, sizeof(double) * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&y, sizeof(double) * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&zo, sizeof(double) * n, st);
    if (e == cudaSuccess) e = cudaMallocAsync(&tw, sizeof(double) * std::max<size_t>(P.blocks.size(), 1) * P.kcap, st);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "alloc simulate");
  }
  if (s == HMLE_OK) {
    FactorArgs F = make_fargs(t, h, f);
    launch_permute_in(st, xd, t->T.perm, n, xp);
    launch_lower_matvec(st, F, t->dp.lr_ids, (int)t->lr_ids.size(), t->dp.mv_row0,
                        t->dp.mv_blocks, P.nleaf, xp, y, tw);
    launch_permute_out(st, y, t->T.perm, n, zo);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(Z, zo, sizeof(double) * n, cudaMemcpyDefault, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) s = cuda_fail(ctx, e, "simulate");
  }
  if (owned) cudaFreeAsync(xd, st);
  if (xp) cudaFreeAsync(xp, st);
  if (y) cudaFreeAsync(y, st);
  if (zo) cudaFreeAsync(zo, st);
  if (tw) cudaFreeAsync(tw, st);
  free_f(st, f);
  delete f;
  hmle_hmatrix_destroy(h);
  return s;
}

hmle_status hmle_matern_eval(hmle_ctx *ctx, double nu, const double *x, int64_t m, double *out) {
  if (!ctx || !x || !out || m < 0) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!(nu > 0) || !(nu <= 20)) return fail(ctx, HMLE_ERR_INVALID_ARG, "nu out of range");
  cudaStream_t st = ctx->st;
  double *tab = nullptr, *xd = nullptr, *od = nullptr;
  bool owned = false;
  CK(cudaMallocAsync(&tab, sizeof(double) * kTableWords, st), "alloc");
  hmle_status s = stage_vec(ctx, x, m, &xd, &owned);
  if (s != HMLE_OK) return s;
  CK(cudaMallocAsync(&od, sizeof(double) * std::max<int64_t>(m, 1), st), "alloc");
  launch_matern_table(st, nu, tab);
  launch_matern_eval(st, tab, xd, m, od);
  CK(cudaGetLastError(), "matern launch");
  CK(cudaMemcpyAsync(out, od, sizeof(double) * m, cudaMemcpyDefault, st), "copy");
  CK(cudaStreamSynchronize(st), "sync");
  cudaFreeAsync(tab, st);
  cudaFreeAsync(od, st);
  if (owned) cudaFreeAsync(xd, st);
  CK(cudaStreamSynchronize(st), "sync");
  return HMLE_OK;
}

hmle_status hmle_cross_matvec(hmle_ctx *ctx, const hmle_tree *t, const hmle_theta *th,
                              const double *locs2, int64_t m, int32_t trans, const double *x,
                              double *y) {
  if (!ctx || !t || !th || !locs2 || !x || !y || m < 1 || (trans != 0 && trans != 1))
    return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!theta_ok(th)) return fail(ctx, HMLE_ERR_INVALID_ARG, "theta out of range");
  cudaStream_t st = ctx->st;
  const int64_t n = t->n, nin = trans ? m : n, nout = trans ? n : m;
  double *tab = nullptr, *l2 = nullptr, *xd = nullptr, *xp = nullptr, *od = nullptr, *oc = nullptr;
  bool lown = false, xown = false;
  hmle_status s = stage_vec(ctx, locs2, m * t->d, &l2, &lown);
  if (s != HMLE_OK) return s;
  s = stage_vec(ctx, x, nin, &xd, &xown);
  if (s != HMLE_OK) { if (lown) cudaFreeAsync(l2, st); return s; }
  CK(cudaMallocAsync(&tab, sizeof(double) * kTableWords, st), "alloc");
  CK(cudaMallocAsync(&od, sizeof(double) * nout, st), "alloc");
  launch_matern_table(st, th->nu, tab);
  if (!trans) {            // y = C21 x: x to cluster order first
    CK(cudaMallocAsync(&xp, sizeof(double) * n, st), "alloc");
    launch_permute_in(st, xd, t->T.perm, n, xp);
    launch_cross_matvec(st, tab, t->T.xyz, n, t->d, l2, m, 1.0 / th->ell, th->sigma2, xp, od);
  } else {                 // y = C12 x: the result back to caller order
    CK(cudaMallocAsync(&oc, sizeof(double) * n, st), "alloc");
    launch_cross_matvec_t(st, tab, t->T.xyz, n, t->d, l2, m, 1.0 / th->ell, th->sigma2, xd, oc);
    launch_permute_out(st, oc, t->T.perm, n, od);
  }
  CK(cudaGetLastError(), "cross matvec launch");
  CK(cudaMemcpyAsync(y, od, sizeof(double) * nout, cudaMemcpyDefault, st), "copy");
  CK(cudaStreamSynchronize(st), "sync");
  for (double *p : {tab, od, xp, oc}) if (p) cudaFreeAsync(p, st);
  if (lown) cudaFreeAsync(l2, st);
  if (xown) cudaFreeAsync(xd, st);
  CK(cudaStreamSynchronize(st), "sync");
  return HMLE_OK;
}

hmle_status hmle_prediction_errors(hmle_ctx *ctx, const hmle_hfactor *ftc, const hmle_hfactor *fac,
                                   const double *locs2, int64_t m, double *mloe, double *mmom,
                                   double *per_point) {
  if (!ctx || !ftc || !fac || !locs2 || m < 1 || m > (1LL << 24) || (!mloe && !mmom && !per_point))
    return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument or m out of range");
  hmle_hfactor *ft = const_cast<hmle_hfactor *>(ftc);
  hmle_hfactor *fa = const_cast<hmle_hfactor *>(fac);
  const hmle_tree *t = ft->h->tree;
  if (fa->h->tree != t) return fail(ctx, HMLE_ERR_INVALID_ARG, "both factors must belong to one tree");
  if (!t->coop) return fail(ctx, HMLE_ERR_NOT_IMPLEMENTED, "the multi-vector sweeps need cooperative launches");
  const hmle_theta tht = ft->h->th, tha = fa->h->th;
  const Plan &P = t->plan;
  cudaStream_t st = ctx->st;
  const int64_t n = t->n, ld = n;
  const int nlr = (int)t->lr_ids.size();
  constexpr int kBlock = 256;    // test locations per round of the sweeps
  constexpr int kMvBlock = 32;   // vectors per launch of the H-matvec (its workspace)
  const int mb = (int)std::min<int64_t>(m, kBlock);
  const int64_t hs = t->mrhs_h, tw = (int64_t)std::max(nlr, 1) * 2 * P.kc;
  double *l2 = nullptr;
  bool lown = false;
  hmle_status s = stage_vec(ctx, locs2, m * t->d, &l2, &lown);
  if (s != HMLE_OK) return s;
  double *tab = nullptr, *V = nullptr, *H = nullptr, *Tw = nullptr, *dots = nullptr;
  unsigned *bar = nullptr;
  cudaError_t e = cudaMallocAsync(&tab, sizeof(double) * 2 * kTableWords, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&V, sizeof(double) * 5 * (size_t)mb * ld, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&H, sizeof(double) * (size_t)mb * hs, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&Tw, sizeof(double) * (size_t)kMvBlock * tw, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&dots, sizeof(double) * 4 * mb, st);
  if (e == cudaSuccess) e = cudaMallocAsync(&bar, 4 * sizeof(unsigned), st);
  if (e == cudaSuccess) e = cudaMemsetAsync(bar, 0, 4 * sizeof(unsigned), st);
  // Ct, Ca: columns c_t(j), c_a(j) of C12 at theta_t and theta_a (cluster
  // order); Lt = C~t^{-1} Ct, La = C~a^{-1} Ca; Y = C~t La (the H-matrix of
  // theta_t)
  double *Ct = V, *Ca = V + (size_t)mb * ld, *Lt = Ca + (size_t)mb * ld, *La = Lt + (size_t)mb * ld,
         *Y = La + (size_t)mb * ld;
  const FactorArgs Ft = make_fargs(t, ft->h, ft), Fa = make_fargs(t, fa->h, fa);
  const hmle_hmatrix *h = ft->h;
  AsmArgs A{};
  A.blocks = t->dp.blocks; A.lr_ids = t->dp.lr_ids; A.xyz = t->T.xyz; A.n = n; A.d = t->d;
  A.tab = h->tab; A.inv_ell = 1.0 / h->th.ell; A.sigma2 = h->th.sigma2; A.tau2 = h->th.tau2;
  A.kc = P.kc; A.uc = h->uc; A.rank_c = h->rank_c; A.cnorm = h->cnorm; A.flags = h->flags;
  A.thd = h->thd; A.Cd = h->Cd; A.b = P.b;
  const CmvLists L{P.nleaf, t->dp.leaf_beg, t->dp.mv_row0, t->dp.mv_blocks, t->dp.mvt_row0,
                   t->dp.mvt_blocks, t->dp.lr_slot};
  if (e == cudaSuccess) {
    launch_matern_table(st, tht.nu, tab);
    launch_matern_table(st, tha.nu, tab + kTableWords);
    e = cudaGetLastError();
  }
  const double vt = tht.sigma2 + tht.tau2, va = tha.sigma2 + tha.tau2;
  std::vector<double> hd(4 * (size_t)mb);
  double sum_loe = 0.0, sum_mom = 0.0;
  unsigned berr = 0;
  for (int64_t j0 = 0; j0 < m && e == cudaSuccess; j0 += mb) {
    const int cnt = (int)std::min<int64_t>(mb, m - j0);
    const size_t bytes = sizeof(double) * (size_t)cnt * ld;
    launch_cross_cols(st, tab, t->T.xyz, n, t->d, l2, j0, cnt, 1.0 / tht.ell, tht.sigma2, Ct, ld);
    launch_cross_cols(st, tab + kTableWords, t->T.xyz, n, t->d, l2, j0, cnt, 1.0 / tha.ell, tha.sigma2, Ca, ld);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(Lt, Ct, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(La, Ca, bytes, cudaMemcpyDeviceToDevice, st);
    if (e == cudaSuccess) e = persistent_solve_multi(st, Ft, t->spm, Lt, ld, H, hs, cnt, bar, false);
    if (e == cudaSuccess) e = persistent_solve_multi(st, Ft, t->spm, Lt, ld, H, hs, cnt, bar, true);
    if (e == cudaSuccess) e = persistent_solve_multi(st, Fa, t->spm, La, ld, H, hs, cnt, bar, false);
    if (e == cudaSuccess) e = persistent_solve_multi(st, Fa, t->spm, La, ld, H, hs, cnt, bar, true);
    for (int c0 = 0; c0 < cnt && e == cudaSuccess; c0 += kMvBlock) {
      const int c = std::min(kMvBlock, cnt - c0);
      launch_cmatvec(st, A, nlr, L, La + (size_t)c0 * ld, Tw, Y + (size_t)c0 * ld, c, ld, tw);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) break;
    launch_col_dots(st, Ct, Lt, n, ld, cnt, dots);
    launch_col_dots(st, Ca, La, n, ld, cnt, dots + mb);
    launch_col_dots(st, La, Ct, n, ld, cnt, dots + 2 * mb);
    launch_col_dots(st, La, Y, n, ld, cnt, dots + 3 * mb);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(hd.data(), dots, sizeof(double) * 4 * mb, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&berr, bar + 2, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess || berr) break;
    for (int jj = 0; jj < cnt; ++jj) {
      const double e_tt = vt - hd[jj];                              // E_t[(Z_t - Z)^2]
      const double e_aa = va - hd[mb + jj];                         // E_a[(Z_a - Z)^2]
      const double e_ta = vt - 2.0 * hd[2 * mb + jj] + hd[3 * mb + jj];   // E_t[(Z_a - Z)^2]
      sum_loe += e_ta / e_tt - 1.0;
      sum_mom += e_aa / e_ta - 1.0;
      if (per_point) {
        per_point[3 * (j0 + jj)] = e_tt;
        per_point[3 * (j0 + jj) + 1] = e_aa;
        per_point[3 * (j0 + jj) + 2] = e_ta;
      }
    }
  }
  for (void *p : {(void *)tab, (void *)V, (void *)H, (void *)Tw, (void *)dots, (void *)bar})
    if (p) cudaFreeAsync(p, st);
  if (lown) cudaFreeAsync(l2, st);
  cudaError_t e2 = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "prediction errors");
  if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "prediction errors");
  if (berr) return fail(ctx, HMLE_ERR_TIMEOUT, "prediction errors: a barrier wait of a sweep ran out");
  if (mloe) *mloe = sum_loe / (double)m;
  if (mmom) *mmom = sum_mom / (double)m;
  return HMLE_OK;
}

hmle_status hmle_profile_select(hmle_ctx *ctx, const char *kernel) {
  if (!ctx) return HMLE_ERR_INVALID_ARG;
  Prof &p = ctx->prof;
  p.kind = -1;
  p.used = 0;
  p.ms = 0.0;
  p.launches = 0;
  p.flops = 0.0;
  p.failed = 0;
  p.first_err = 0;
  if (!kernel) return HMLE_OK;
  for (int k = 0; k < KK_COUNT; ++k)
    if (std::strcmp(kernel, kKernelNames[k]) == 0) p.kind = k;
  return p.kind >= 0 ? HMLE_OK : fail(ctx, HMLE_ERR_INVALID_ARG, "unknown kernel name");
}

hmle_status hmle_profile_read(hmle_ctx *ctx, double *ms, int64_t *launches, double *flops) {
  if (!ctx) return HMLE_ERR_INVALID_ARG;
  if (ms) *ms = ctx->prof.ms;
  if (launches) *launches = ctx->prof.launches;
  if (flops) *flops = ctx->prof.flops;
  return HMLE_OK;
}

hmle_status hmle_phase_work(hmle_ctx *ctx, const hmle_hfactor *f, double *asm_flops,
                            double *solve_bytes) {
  if (!ctx || !f || !f->h) return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  const hmle_hmatrix *h = f->h;
  const hmle_tree *t = h->tree;
  const Plan &P = t->plan;
  const size_t nb = P.blocks.size();
  std::vector<int32_t> rc(nb), rl(nb);
  CK(cudaMemcpyAsync(rc.data(), h->rank_c, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, ctx->st), "ranks");
  CK(cudaMemcpyAsync(rl.data(), f->rank_l, sizeof(int32_t) * nb, cudaMemcpyDeviceToHost, ctx->st), "ranks");
  CK(cudaStreamSynchronize(ctx->st), "sync");
  const double e = 3.0 * t->d + 68.0;   // flops per Matern entry
  double fa = 0.0, words = 0.0;
  for (size_t x = 0; x < nb; ++x) {
    const BlockDesc &B = P.blocks[x];
    const double m = B.rend - B.rbeg, p = B.cend - B.cbeg;
    if (B.kind == kDense) {
      fa += m * p * e;
      words += (B.rbeg == B.cbeg) ? m * (m + 1.0) / 2.0 : m * p;
    } else {
      const double k = rc[x];
      fa += (m + p) * (k * e + k * (k - 1.0));
      words += (m + p) * rl[x];
    }
  }
  if (asm_flops) *asm_flops = fa;
  if (solve_bytes) *solve_bytes = 2.0 * 8.0 * words;
  return HMLE_OK;
}

// --- MLE (Sec. 2; transform of Sec. 5) ----------------------------------
static void to_theta(const double x[4], hmle_theta *t) {
  double sigma = 2.0 / std::pow(1.1, x[0]);
  t->ell = 1.0 / std::pow(1.5, x[1]);
  t->nu = 1.0 / std::pow(1.2, x[2]);
  double tau = 1.0 / std::pow(2.0, x[3]);
  t->sigma2 = sigma * sigma;
  t->tau2 = tau * tau;
}

static void from_theta(const hmle_theta *t, double x[4]) {
  x[0] = -std::log(std::sqrt(t->sigma2) / 2.0) / std::log(1.1);
  x[1] = -std::log(t->ell) / std::log(1.5);
  x[2] = -std::log(t->nu) / std::log(1.2);
  x[3] = -std::log(std::sqrt(t->tau2)) / std::log(2.0);
}

hmle_status hmle_theta_to_x(const hmle_theta *theta, double x[4]) {
  if (!theta || !x || !theta_ok(theta) || !(theta->sigma2 > 0.0) || !(theta->tau2 > 0.0))
    return HMLE_ERR_INVALID_ARG;
  from_theta(theta, x);
  return HMLE_OK;
}

hmle_status hmle_x_to_theta(const double x[4], hmle_theta *theta) {
  if (!theta || !x) return HMLE_ERR_INVALID_ARG;
  for (int k = 0; k < 4; ++k)
    if (!std::isfinite(x[k])) return HMLE_ERR_INVALID_ARG;
  to_theta(x, theta);
  return theta_ok(theta) ? HMLE_OK : HMLE_ERR_INVALID_ARG;
}

}  // extern "C"

namespace {

// Nelder-Mead (reflection 1, expansion 2, contraction 1/2, shrink 1/2) in D
// transformed coordinates.  Each iteration evaluates its four candidates
// (reflection, expansion, outside and inside contraction) together as one
// batch and then applies the usual acceptance rules; nev counts the
// evaluations the rules use.  Stops when the simplex's f-spread <= ftol and
// x-spread <= xtol (Sec. 2 threshold) or after max_iter iterations.  fbatch(xs,
// k, fv): f at k points (+inf where undefined).  On return X[0] is the best
// vertex; the result says whether the tolerance was met.
template <int D, class FB>
bool nelder_mead(FB fbatch, const double x0[D], const double step[D], const hmle_fit_opts &fo,
                 const hmle_status &hard, double (&X)[D + 1][D], double (&Fv)[D + 1], int &it,
                 int &nev) {
  for (int j = 0; j < D; ++j) X[0][j] = x0[j];
  for (int i = 1; i <= D; ++i) {
    for (int j = 0; j < D; ++j) X[i][j] = X[0][j];
    X[i][i - 1] += step[i - 1];
  }
  fbatch(X, D + 1, Fv);
  nev = D + 1;
  it = 0;
  while (hard == HMLE_OK) {
    // stable order by f
    int ord[D + 1];
    for (int i = 0; i <= D; ++i) ord[i] = i;
    std::stable_sort(ord, ord + D + 1, [&](int a, int b) { return Fv[a] < Fv[b]; });
    double Xs[D + 1][D], Fs[D + 1];
    for (int i = 0; i <= D; ++i) { Fs[i] = Fv[ord[i]]; for (int j = 0; j < D; ++j) Xs[i][j] = X[ord[i]][j]; }
    std::memcpy(X, Xs, sizeof(X));
    std::memcpy(Fv, Fs, sizeof(Fv));
    double fs = 0, xs = 0;
    for (int i = 1; i <= D; ++i) {
      fs = std::max(fs, std::fabs(Fv[i] - Fv[0]));
      for (int j = 0; j < D; ++j) xs = std::max(xs, std::fabs(X[i][j] - X[0][j]));
    }
    if (std::isfinite(Fv[D]) && fs <= fo.ftol && xs <= fo.xtol) return true;
    if (it >= fo.max_iter) return false;
    ++it;
    double c[D];
    for (int j = 0; j < D; ++j) c[j] = 0.0;
    for (int i = 0; i < D; ++i) for (int j = 0; j < D; ++j) c[j] += X[i][j] / D;
    double cand[4][D], fc[4];
    for (int j = 0; j < D; ++j) {
      const double d = c[j] - X[D][j];
      cand[0][j] = c[j] + d;
      cand[1][j] = c[j] + 2.0 * d;
      cand[2][j] = c[j] + 0.5 * d;
      cand[3][j] = c[j] - 0.5 * d;
    }
    fbatch(cand, 4, fc);
    if (hard != HMLE_OK) return false;
    const double fr = fc[0];
    ++nev;
    bool shrink = false;
    if (Fv[0] <= fr && fr < Fv[D - 1]) {
      std::memcpy(X[D], cand[0], sizeof(cand[0])); Fv[D] = fr;
    } else if (fr < Fv[0]) {
      ++nev;
      if (fc[1] < fr) { std::memcpy(X[D], cand[1], sizeof(cand[1])); Fv[D] = fc[1]; }
      else { std::memcpy(X[D], cand[0], sizeof(cand[0])); Fv[D] = fr; }
    } else if (fr < Fv[D]) {
      ++nev;
      if (fc[2] <= fr) { std::memcpy(X[D], cand[2], sizeof(cand[2])); Fv[D] = fc[2]; }
      else shrink = true;
    } else {
      ++nev;
      if (fc[3] < Fv[D]) { std::memcpy(X[D], cand[3], sizeof(cand[3])); Fv[D] = fc[3]; }
      else shrink = true;
    }
    if (shrink) {
      for (int i = 1; i <= D; ++i)
        for (int j = 0; j < D; ++j) X[i][j] = X[0][j] + 0.5 * (X[i][j] - X[0][j]);
      fbatch(&X[1], D, &Fv[1]);
      nev += D;
    }
  }
  return false;
}

template <int D>
hmle_status nelder_mead_host(hmle_objective f, void *user, const double *x0, const double *step,
                             const hmle_fit_opts &fo, double *x_best, double *f_best,
                             int32_t *n_iter, int32_t *n_evals) {
  double st[D], x[D];
  for (int j = 0; j < D; ++j) {
    x[j] = x0[j];
    st[j] = step ? step[j] : 1.0;
  }
  const hmle_status hard = HMLE_OK;
  auto fbatch = [&](const double (*xs)[D], int k, double *fv) {
    for (int i = 0; i < k; ++i) {
      const double v = f(xs[i], D, user);
      fv[i] = std::isnan(v) ? INFINITY : v;
    }
  };
  double X[D + 1][D], Fv[D + 1];
  int it = 0, nev = 0;
  const bool conv = nelder_mead<D>(fbatch, x, st, fo, hard, X, Fv, it, nev);
  for (int j = 0; j < D; ++j) x_best[j] = X[0][j];
  if (f_best) *f_best = Fv[0];
  if (n_iter) *n_iter = it;
  if (n_evals) *n_evals = nev;
  return conv ? HMLE_OK : HMLE_ERR_NOT_CONVERGED;
}

}  // namespace

extern "C" {

hmle_status hmle_nelder_mead(int32_t dim, hmle_objective f, void *user, const double *x0,
                             const double *step, const hmle_fit_opts *fo_in, double *x_best,
                             double *f_best, int32_t *n_iter, int32_t *n_evals) {
  if (!f || !x0 || !x_best) return HMLE_ERR_INVALID_ARG;
  for (int j = 0; j < dim; ++j)
    if (!std::isfinite(x0[j]) || (step && !std::isfinite(step[j]))) return HMLE_ERR_INVALID_ARG;
  hmle_fit_opts fo;
  if (fo_in) fo = *fo_in; else hmle_fit_opts_default(&fo);
  switch (dim) {
    case 1: return nelder_mead_host<1>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 2: return nelder_mead_host<2>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 3: return nelder_mead_host<3>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 4: return nelder_mead_host<4>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 5: return nelder_mead_host<5>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 6: return nelder_mead_host<6>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 7: return nelder_mead_host<7>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    case 8: return nelder_mead_host<8>(f, user, x0, step, fo, x_best, f_best, n_iter, n_evals);
    default: return HMLE_ERR_INVALID_ARG;
  }
}

hmle_status hmle_fit(hmle_ctx *ctx, const hmle_tree *t, const double *Z, const hmle_theta *theta0,
                     const hmle_fit_opts *fo_in, hmle_theta *theta_hat, double *ll_hat,
                     int32_t *n_iter, int32_t *n_evals) {
  if (!ctx || !t || !Z || !theta0 || !theta_hat || !ll_hat)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!theta_ok(theta0) || theta0->sigma2 <= 0 || theta0->tau2 <= 0)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "theta0 must have sigma2 > 0 and tau2 > 0");
  hmle_fit_opts fo;
  if (fo_in) fo = *fo_in; else hmle_fit_opts_default(&fo);
  double step[4];
  bool allzero = true;
  for (int i = 0; i < 4; ++i) { step[i] = fo.step[i]; allzero &= (step[i] == 0.0); }
  if (allzero) for (int i = 0; i < 4; ++i) step[i] = 1.0;
  double *zd = nullptr;
  bool owned = false;
  hmle_status s = stage_vec(ctx, Z, t->n, &zd, &owned);
  if (s != HMLE_OK) return s;
  hmle_status hard = HMLE_OK;
  hmle_tree *tt = const_cast<hmle_tree *>(t);
  // -L at several transformed points, evaluated concurrently
  auto fbatch = [&](const double (*xs)[4], int k, double *fv) {
    hmle_theta th[5];
    int idx[5], m = 0;
    for (int i = 0; i < k; ++i) {
      to_theta(xs[i], &th[m]);
      if (theta_ok(&th[m])) { idx[m] = i; ++m; }
      fv[i] = INFINITY;
    }
    if (m == 0) return;
    double ll[5];
    int32_t st[5];
    hmle_status r = batch_eval(ctx, tt, th, m, zd, m, ll, st, nullptr, nullptr);
    if (r != HMLE_OK) { hard = r; return; }
    for (int j = 0; j < m; ++j)
      fv[idx[j]] = (st[j] == HMLE_OK) ? -ll[j] : INFINITY;
  };
  double x0[4], X[5][4], Fv[5];
  from_theta(theta0, x0);
  int it = 0, nev = 0;
  const bool conv = nelder_mead<4>(fbatch, x0, step, fo, hard, X, Fv, it, nev);
  if (owned) cudaFreeAsync(zd, ctx->st);
  cudaStreamSynchronize(ctx->st);
  if (hard != HMLE_OK) return hard;
  to_theta(X[0], theta_hat);
  *ll_hat = -Fv[0];
  if (n_iter) *n_iter = it;
  if (n_evals) *n_evals = nev;
  return conv ? HMLE_OK : fail(ctx, HMLE_ERR_NOT_CONVERGED, "max_iter reached");
}

hmle_status hmle_fit_profiled(hmle_ctx *ctx, const hmle_tree *t, const double *Z,
                              const hmle_theta *theta0, const hmle_fit_opts *fo_in,
                              hmle_theta *theta_hat, double *ll_hat, int32_t *n_iter,
                              int32_t *n_evals) {
  if (!ctx || !t || !Z || !theta0 || !theta_hat || !ll_hat)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "null argument");
  if (!theta_ok(theta0) || theta0->sigma2 <= 0 || theta0->tau2 <= 0)
    return fail(ctx, HMLE_ERR_INVALID_ARG, "theta0 must have sigma2 > 0 and tau2 > 0");
  hmle_fit_opts fo;
  if (fo_in) fo = *fo_in; else hmle_fit_opts_default(&fo);
  // coordinates (ell0, nu0, r0): ell = 1 / 1.5^ell0, nu = 1 / 1.2^nu0 (Sec. 5)
  // and the nugget-to-variance ratio rho = tau2 / sigma2 = (1 / 2^r0)^2
  double step[3];
  bool allzero = true;
  for (int i = 0; i < 3; ++i) { step[i] = fo.step[i + 1]; allzero &= (step[i] == 0.0); }
  if (allzero) for (int i = 0; i < 3; ++i) step[i] = 1.0;
  const double n = (double)t->n;
  auto to_unit = [](const double x[3], hmle_theta *th) {   // sigma2 = 1, tau2 = rho
    th->ell = 1.0 / std::pow(1.5, x[0]);
    th->nu = 1.0 / std::pow(1.2, x[1]);
    th->sigma2 = 1.0;
    const double r = 1.0 / std::pow(2.0, x[2]);
    th->tau2 = r * r;
  };
  double *zd = nullptr;
  bool owned = false;
  hmle_status s = stage_vec(ctx, Z, t->n, &zd, &owned);
  if (s != HMLE_OK) return s;
  hmle_status hard = HMLE_OK;
  hmle_tree *tt = const_cast<hmle_tree *>(t);
  // -L_p: with C = sigma2 R_rho, log|C| = n log sigma2 + log|R_rho| and
  // Z^T C^-1 Z = q / sigma2 are maximised over sigma2 by sigma2 = q / n, so
  // L_p = -n/2 log(2 pi) - n/2 log(q / n) - 1/2 log|R_rho| - n/2
  auto fbatch = [&](const double (*xs)[3], int k, double *fv) {
    hmle_theta th[5];
    int idx[5], m = 0;
    for (int i = 0; i < k; ++i) {
      to_unit(xs[i], &th[m]);
      if (theta_ok(&th[m]) && std::isfinite(th[m].tau2)) { idx[m] = i; ++m; }
      fv[i] = INFINITY;
    }
    if (m == 0) return;
    double ll[5], ld[5], q[5];
    int32_t st[5];
    hmle_status r = batch_eval(ctx, tt, th, m, zd, m, ll, st, ld, q);
    if (r != HMLE_OK) { hard = r; return; }
    for (int j = 0; j < m; ++j)
      fv[idx[j]] = (st[j] == HMLE_OK && q[j] > 0.0)
                       ? 0.5 * n * std::log(2.0 * M_PI) + 0.5 * n * std::log(q[j] / n) +
                             0.5 * ld[j] + 0.5 * n
                       : INFINITY;
  };
  double x0[3] = {-std::log(theta0->ell) / std::log(1.5), -std::log(theta0->nu) / std::log(1.2),
                  -std::log(std::sqrt(theta0->tau2 / theta0->sigma2)) / std::log(2.0)};
  double X[4][3], Fv[4];
  int it = 0, nev = 0;
  const bool conv = nelder_mead<3>(fbatch, x0, step, fo, hard, X, Fv, it, nev);
  hmle_status out = HMLE_OK;
  if (hard == HMLE_OK) {
    // sigma2 of the optimum: one more evaluation at the best point
    hmle_theta th;
    to_unit(X[0], &th);
    double ll, ld, q;
    int32_t st;
    out = batch_eval(ctx, tt, &th, 1, zd, 1, &ll, &st, &ld, &q);
    if (out == HMLE_OK && st == HMLE_OK) {
      const double s2 = q / n;
      theta_hat->ell = th.ell;
      theta_hat->nu = th.nu;
      theta_hat->sigma2 = s2;
      theta_hat->tau2 = th.tau2 * s2;
      *ll_hat = -Fv[0];
    } else if (out == HMLE_OK) {
      out = (hmle_status)st;
    }
  }
  if (owned) cudaFreeAsync(zd, ctx->st);
  cudaStreamSynchronize(ctx->st);
  if (hard != HMLE_OK) return hard;
  if (out != HMLE_OK) return out;
  if (n_iter) *n_iter = it;
  if (n_evals) *n_evals = nev + 1;
  return conv ? HMLE_OK : fail(ctx, HMLE_ERR_NOT_CONVERGED, "max_iter reached");
}

}  // extern "C"
