// a15: the autotuner of the batched form (no counterpart in the paper).
//
// For one point set and one theta it times hmle_loglik_batch over a small
// grid of leaf sizes (the tile of the leaf sweep: dense blocks are b x b,
// every step of the sweep handles one leaf), concurrencies (evaluations in
// flight) and batch sizes (evaluations served by one launch of each sweep
// kernel; the sub-batches of a concurrency run side by side on their own
// streams), and returns the combination with the most evaluations per
// second.  It uses only the public C ABI.
#include <cuda_runtime.h>

#include <chrono>
#include <cstring>
#include <vector>

#include "../../include/hmle.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

}  // namespace

extern "C" hmle_status hmle_autotune(hmle_ctx *ctx, const double *locs, int64_t n, int32_t d,
                                     const hmle_opts *base, const hmle_theta *theta,
                                     const double *Z, int32_t max_concurrency,
                                     hmle_tune_result *best, hmle_tune_result *trials,
                                     int32_t max_trials, int32_t *ntrials) {
  if (!ctx || !locs || !base || !theta || !Z || !best || n <= 0) return HMLE_ERR_INVALID_ARG;
  if (max_concurrency <= 0) max_concurrency = 16;
  if (max_concurrency > 64) max_concurrency = 64;
  const int32_t leaves[] = {32, 64, 128};
  std::memset(best, 0, sizeof(*best));
  int32_t nt = 0;
  hmle_status first = HMLE_OK;
  for (int32_t leaf : leaves) {
    if ((int64_t)leaf > n) continue;
    hmle_opts o = *base;
    o.leaf_size = leaf;
    hmle_tree *t = nullptr;
    hmle_status s = hmle_build_tree(ctx, locs, n, d, &o, &t);
    if (s != HMLE_OK) { if (first == HMLE_OK) first = s; continue; }
    double prev = 0.0;
    bool failed = false;
    for (int32_t c = 1; c <= max_concurrency && !failed; c *= 2) {
      std::vector<hmle_theta> th(c, *theta);
      std::vector<double> ll(c);
      std::vector<int32_t> st(c);
      double best_c = 0.0;
      int32_t last_bs = 0;
      for (int32_t div = 1; div <= 4; div *= 2) {   // evaluations per launch: c, c / 2, c / 4
        const int32_t bs = c / div > 0 ? c / div : 1;
        if (bs == last_bs) continue;
        last_bs = bs;
        hmle_tree_set_batch_size(t, bs);
        // warm-up: allocates the c buffers and captures their graphs
        s = hmle_loglik_batch(ctx, t, th.data(), c, Z, c, ll.data(), st.data());
        double t0 = now_s();
        if (s == HMLE_OK) s = hmle_loglik_batch(ctx, t, th.data(), c, Z, c, ll.data(), st.data());
        const double dt = now_s() - t0;
        bool ok = (s == HMLE_OK);
        for (int32_t k = 0; k < c && ok; ++k) ok = (st[k] == HMLE_OK);
        if (!ok) {   // this candidate fails (e.g. a rank overflow): record it, try the next leaf size
          if (first == HMLE_OK) first = (s != HMLE_OK ? s : (hmle_status)st[0]);
          cudaGetLastError();
          hmle_tune_result r{leaf, c, 0.0, 0, bs};
          if (trials && nt < max_trials) trials[nt] = r;
          ++nt;
          failed = true;
          break;
        }
        hmle_tune_result r{leaf, c, dt > 0.0 ? c / dt : 0.0, 0, bs};
        if (trials && nt < max_trials) trials[nt] = r;
        ++nt;
        if (r.evals_per_s > best->evals_per_s) *best = r;
        best_c = r.evals_per_s > best_c ? r.evals_per_s : best_c;
      }
      if (failed || best_c < 1.05 * prev) break;   // saturated
      prev = best_c;
    }
    hmle_tree_destroy(t);
  }
  best->trials = nt;
  if (ntrials) *ntrials = nt;
  if (best->leaf_size == 0) return first != HMLE_OK ? first : HMLE_ERR_INVALID_ARG;
  return HMLE_OK;
}
