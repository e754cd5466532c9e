// a1-a2 (Sec. 2, recursive block partition): geometric cluster tree and
// block tree on the device.
//
// Cluster tree: a balanced binary tree over the points.  A cluster is a
// contiguous range of the cluster-order permutation; it is split at its
// median along the longest side of its bounding box (ties to the lowest
// axis), the left child taking floor(size / 2) points.  One level is one
// stable LSD radix sort of all points by (cluster index, coordinate along
// the cluster's axis quantised to 32 bits within its box): the cluster
// index is already sorted, so this is a segmented sort.  Points whose
// quantised coordinates tie keep their previous order.
//
// Block tree: breadth-first over levels from (root, root).  A pair (i, j),
// i >= j, of clusters of one level is admissible when i != j and
// min(diam_i, diam_j) <= eta * dist(i, j) (Euclidean diameter and distance
// of the bounding boxes); admissible pairs become low-rank blocks, pairs at
// the leaf level dense blocks, and other pairs split into their 3 (i == j)
// or 4 children in the lower triangle.  Every level is compacted with an
// exclusive scan, so the output order is deterministic.
#include <cuda_runtime.h>

#include "common.cuh"
#include "tree.cuh"

namespace hmle {

namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 8;
constexpr int kTile = kSortThreads * kSortItems;

// bounding box of clusters [c0, c0 + nc) of one level; ranges given by beg/end
__global__ void k_bbox(const double *__restrict__ xyz, int64_t n, int d,
                       const int32_t *__restrict__ beg, const int32_t *__restrict__ end,
                       int32_t c0, double *__restrict__ box) {
  __shared__ double red[32];
  const int c = c0 + blockIdx.x;
  const int b = beg[c], e = end[c];
  for (int k = 0; k < d; ++k) {
    double lo = INFINITY, hi = -INFINITY;
    for (int i = b + threadIdx.x; i < e; i += blockDim.x) {
      double v = xyz[k * n + i];
      lo = fmin(lo, v);
      hi = fmax(hi, v);
    }
    // min via negated sum trick is not exact; use warp min/max
    for (int o = 16; o > 0; o >>= 1) {
      lo = fmin(lo, __shfl_xor_sync(0xffffffffu, lo, o));
      hi = fmax(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    __syncthreads();
    if ((threadIdx.x & 31) == 0) { red[threadIdx.x >> 5] = lo; red[16 + (threadIdx.x >> 5)] = hi; }
    __syncthreads();
    if (threadIdx.x == 0) {
      const int nw = blockDim.x >> 5;
      double L = red[0], H = red[16];
      for (int w = 1; w < nw; ++w) { L = fmin(L, red[w]); H = fmax(H, red[16 + w]); }
      box[(int64_t)c * 6 + k] = L;
      box[(int64_t)c * 6 + 3 + k] = H;
    }
  }
}

// sort keys of one level: key = (cluster index within the level) << 32 | q
__global__ void k_level_keys(const double *__restrict__ xyz, int64_t n, int d,
                             const int32_t *__restrict__ clus_of_pos,
                             const double *__restrict__ box, int32_t c0,
                             uint64_t *__restrict__ key, int32_t *__restrict__ val) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int c = clus_of_pos[i];               // heap id of the cluster holding position i
  const double *bx = box + (int64_t)c * 6;
  int ax = 0;
  double ext = bx[3] - bx[0];
  for (int k = 1; k < d; ++k) {
    double e = bx[3 + k] - bx[k];
    if (e > ext) { ext = e; ax = k; }
  }
  double v = xyz[ax * n + i];
  uint32_t q = 0;
  if (ext > 0.0) {
    double f = (v - bx[ax]) / ext;
    f = fmin(fmax(f, 0.0), 1.0);
    q = (uint32_t)(f * 4294967295.0);
  }
  key[i] = ((uint64_t)(c - c0) << 32) | q;
  val[i] = (int32_t)i;
}

// per-tile histogram of one 8-bit digit; hist is digit-major: hist[dg * ntiles + tile]
__global__ void k_radix_hist(const uint64_t *__restrict__ key, int64_t n, int shift,
                             int32_t *__restrict__ hist, int ntiles) {
  __shared__ int32_t h[256];
  for (int t = threadIdx.x; t < 256; t += blockDim.x) h[t] = 0;
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + (int64_t)it * kSortThreads + threadIdx.x;
    if (i < n) atomicAdd(&h[(key[i] >> shift) & 255], 1);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < 256; t += blockDim.x) hist[(int64_t)t * ntiles + blockIdx.x] = h[t];
}

// stable scatter: ranks within a tile follow the input order
__global__ void k_radix_scatter(const uint64_t *__restrict__ key, const int32_t *__restrict__ val,
                                int64_t n, int shift, const int32_t *__restrict__ offs,
                                int ntiles, uint64_t *__restrict__ key2,
                                int32_t *__restrict__ val2) {
  __shared__ int32_t cnt[256];
  __shared__ int32_t base_of[256];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int t = threadIdx.x; t < 256; t += blockDim.x) {
    cnt[t] = 0;
    base_of[t] = offs[(int64_t)t * ntiles + blockIdx.x];
  }
  __syncthreads();
  int64_t base = (int64_t)blockIdx.x * kTile;
  for (int it = 0; it < kSortItems; ++it) {
    int64_t i = base + (int64_t)it * kSortThreads + threadIdx.x;
    bool ok = i < n;
    uint64_t k = ok ? key[i] : 0;
    int dg = ok ? (int)((k >> shift) & 255) : 256 + lane;  // unique dummy digits
    unsigned peers = __match_any_sync(0xffffffffu, dg);
    int rank = __popc(peers & ((1u << lane) - 1u));
    int total = __popc(peers);
    int leader = __ffs(peers) - 1;
    // warps in order, so that earlier elements get lower ranks
    for (int w = 0; w < kSortThreads / 32; ++w) {
      if (wid == w && ok) {
        int pos = base_of[dg] + cnt[dg] + rank;
        key2[pos] = k;
        val2[pos] = val[i];
      }
      __syncwarp();
      if (wid == w && ok && lane == leader) cnt[dg] += total;
      __syncthreads();
    }
  }
}

// single-block exclusive scan of m int32 values in place
__global__ void k_scan_excl(int32_t *__restrict__ a, int64_t m) {
  __shared__ int32_t part[1024];
  const int T = blockDim.x;
  int64_t per = (m + T - 1) / T;
  int64_t lo = threadIdx.x * per, hi = lo + per < m ? lo + per : m;
  int32_t s = 0;
  for (int64_t i = lo; i < hi; ++i) s += a[i];
  part[threadIdx.x] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int32_t run = 0;
    for (int t = 0; t < T; ++t) { int32_t v = part[t]; part[t] = run; run += v; }
  }
  __syncthreads();
  int32_t run = part[threadIdx.x];
  for (int64_t i = lo; i < hi; ++i) { int32_t v = a[i]; a[i] = run; run += v; }
}

__global__ void k_gather_coords(const double *__restrict__ xyz_in, int64_t n, int d,
                                const int32_t *__restrict__ src, double *__restrict__ xyz_out,
                                const int32_t *__restrict__ perm_in, int32_t *__restrict__ perm_out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int32_t s = src[i];
  for (int k = 0; k < d; ++k) xyz_out[k * n + i] = xyz_in[k * n + s];
  perm_out[i] = perm_in[s];
}

__global__ void k_fill_cluster_of_pos(const int32_t *__restrict__ beg, const int32_t *__restrict__ end,
                                      int32_t c0, int32_t nc, int32_t *__restrict__ cop) {
  int c = c0 + blockIdx.x;
  if (blockIdx.x >= nc) return;
  for (int i = beg[c] + threadIdx.x; i < end[c]; i += blockDim.x) cop[i] = c;
}

__global__ void k_iota(int32_t *a, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) a[i] = (int32_t)i;
}

// rows (n x d, row-major) -> SoA; flags non-finite coordinates
__global__ void k_to_soa(const double *__restrict__ rows, int64_t n, int d,
                         double *__restrict__ xyz, int *__restrict__ bad) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  for (int k = 0; k < d; ++k) {
    double v = rows[i * d + k];
    if (!isfinite(v)) atomicOr(bad, 1);
    xyz[k * n + i] = v;
  }
}

// --- block tree ---------------------------------------------------------

__device__ __forceinline__ bool admissible(const double *__restrict__ box, int d, int hi, int hj,
                                           double eta) {
  const double *a = box + (int64_t)hi * 6, *b = box + (int64_t)hj * 6;
  double da = 0.0, db = 0.0, dist = 0.0;
  for (int k = 0; k < d; ++k) {
    double ea = a[3 + k] - a[k], eb = b[3 + k] - b[k];
    da = fma(ea, ea, da);
    db = fma(eb, eb, db);
    double g = fmax(0.0, fmax(a[k] - b[3 + k], b[k] - a[3 + k]));
    dist = fma(g, g, dist);
  }
  return sqrt(fmin(da, db)) <= eta * sqrt(dist);
}

// classify frontier pairs: out_cnt = #emitted blocks (0/1), ch_cnt = #children
__global__ void k_bt_classify(const int2 *__restrict__ fr, int32_t nf, int level, int depth, int d,
                              const double *__restrict__ box, double eta,
                              int32_t *__restrict__ out_cnt, int32_t *__restrict__ ch_cnt,
                              int8_t *__restrict__ kind) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  int2 p = fr[t];
  int base = (1 << level) - 1;
  int8_t k;
  if (p.x != p.y && admissible(box, d, base + p.x, base + p.y, eta)) {
    k = 1; out_cnt[t] = 1; ch_cnt[t] = 0;
  } else if (level == depth) {
    k = 0; out_cnt[t] = 1; ch_cnt[t] = 0;
  } else {
    k = 2; out_cnt[t] = 0; ch_cnt[t] = (p.x == p.y) ? 3 : 4;
  }
  kind[t] = k;
}

__global__ void k_bt_emit(const int2 *__restrict__ fr, int32_t nf, int level,
                          const int8_t *__restrict__ kind, const int32_t *__restrict__ out_off,
                          const int32_t *__restrict__ ch_off, int4 *__restrict__ blocks,
                          int32_t blocks_base, int2 *__restrict__ next) {
  int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nf) return;
  int2 p = fr[t];
  int8_t k = kind[t];
  if (k < 2) {
    blocks[blocks_base + out_off[t]] = make_int4(level, p.x, p.y, (int)k);
  } else {
    int o = ch_off[t];
    int i0 = 2 * p.x, j0 = 2 * p.y;
    if (p.x == p.y) {
      next[o + 0] = make_int2(i0, j0);
      next[o + 1] = make_int2(i0 + 1, j0);
      next[o + 2] = make_int2(i0 + 1, j0 + 1);
    } else {
      next[o + 0] = make_int2(i0, j0);
      next[o + 1] = make_int2(i0, j0 + 1);
      next[o + 2] = make_int2(i0 + 1, j0);
      next[o + 3] = make_int2(i0 + 1, j0 + 1);
    }
  }
}

inline unsigned nblk(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

// --- host orchestration ---------------------------------------------------

std::string tree_build_device(cudaStream_t st, const double *rows_dev, int64_t n, int d,
                              int depth, const std::vector<int32_t> &cl_beg,
                              const std::vector<int32_t> &cl_end, double eta,
                              DeviceTree &T, std::vector<int4> &blocks_out) {
  auto ck = [](cudaError_t e) -> std::string {
    return e == cudaSuccess ? std::string() : std::string(cudaGetErrorString(e));
  };
  std::string err;
  const int ncl = (int)cl_beg.size();
  int32_t *d_beg = nullptr, *d_end = nullptr, *d_cop = nullptr, *d_val = nullptr,
          *d_val2 = nullptr, *d_hist = nullptr, *d_perm2 = nullptr, *d_bad = nullptr;
  uint64_t *d_key = nullptr, *d_key2 = nullptr;
  double *d_xyz2 = nullptr;
  const int64_t ntiles = (n + kTile - 1) / kTile;
#define TRY(x) do { err = ck(x); if (!err.empty()) goto done; } while (0)
  TRY(cudaMallocAsync(&T.xyz, sizeof(double) * 3 * n, st));
  TRY(cudaMallocAsync(&T.perm, sizeof(int32_t) * n, st));
  TRY(cudaMallocAsync(&T.box, sizeof(double) * 6 * ncl, st));
  TRY(cudaMallocAsync(&d_beg, sizeof(int32_t) * ncl, st));
  TRY(cudaMallocAsync(&d_end, sizeof(int32_t) * ncl, st));
  TRY(cudaMallocAsync(&d_cop, sizeof(int32_t) * n, st));
  TRY(cudaMallocAsync(&d_val, sizeof(int32_t) * n, st));
  TRY(cudaMallocAsync(&d_val2, sizeof(int32_t) * n, st));
  TRY(cudaMallocAsync(&d_perm2, sizeof(int32_t) * n, st));
  TRY(cudaMallocAsync(&d_key, sizeof(uint64_t) * n, st));
  TRY(cudaMallocAsync(&d_key2, sizeof(uint64_t) * n, st));
  TRY(cudaMallocAsync(&d_xyz2, sizeof(double) * 3 * n, st));
  TRY(cudaMallocAsync(&d_hist, sizeof(int32_t) * 256 * ntiles, st));
  TRY(cudaMallocAsync(&d_bad, sizeof(int32_t), st));
  TRY(cudaMemsetAsync(d_bad, 0, sizeof(int32_t), st));
  TRY(cudaMemsetAsync(T.box, 0, sizeof(double) * 6 * ncl, st));
  TRY(cudaMemcpyAsync(d_beg, cl_beg.data(), sizeof(int32_t) * ncl, cudaMemcpyHostToDevice, st));
  TRY(cudaMemcpyAsync(d_end, cl_end.data(), sizeof(int32_t) * ncl, cudaMemcpyHostToDevice, st));
  k_to_soa<<<nblk(n, 256), 256, 0, st>>>(rows_dev, n, d, T.xyz, d_bad);
  k_iota<<<nblk(n, 256), 256, 0, st>>>(T.perm, n);
  for (int l = 0; l <= depth; ++l) {
    const int c0 = (1 << l) - 1, nc = 1 << l;
    k_bbox<<<nc, 256, 0, st>>>(T.xyz, n, d, d_beg, d_end, c0, T.box);
    if (l == depth) break;
    k_fill_cluster_of_pos<<<nc, 256, 0, st>>>(d_beg, d_end, c0, nc, d_cop);
    k_level_keys<<<nblk(n, 256), 256, 0, st>>>(T.xyz, n, d, d_cop, T.box, c0, d_key, d_val);
    const int bits = 32 + l;
    for (int shift = 0; shift < bits; shift += 8) {
      k_radix_hist<<<(unsigned)ntiles, kSortThreads, 0, st>>>(d_key, n, shift, d_hist, (int)ntiles);
      k_scan_excl<<<1, 1024, 0, st>>>(d_hist, 256 * ntiles);
      k_radix_scatter<<<(unsigned)ntiles, kSortThreads, 0, st>>>(d_key, d_val, n, shift, d_hist,
                                                                (int)ntiles, d_key2, d_val2);
      std::swap(d_key, d_key2);
      std::swap(d_val, d_val2);
    }
    k_gather_coords<<<nblk(n, 256), 256, 0, st>>>(T.xyz, n, d, d_val, d_xyz2, T.perm, d_perm2);
    std::swap(T.xyz, d_xyz2);
    std::swap(T.perm, d_perm2);
  }
  TRY(cudaGetLastError());
  {
    int32_t bad = 0;
    TRY(cudaMemcpyAsync(&bad, d_bad, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));
    if (bad) { err = "non-finite coordinate in locs"; goto done; }
  }
  // --- block tree
  {
    std::vector<int2> hfront(1, make_int2(0, 0));
    int2 *d_fr = nullptr, *d_next = nullptr;
    int32_t *d_oc = nullptr, *d_cc = nullptr;
    int8_t *d_kind = nullptr;
    int4 *d_blocks = nullptr;
    int32_t nf = 1;
    std::vector<int4> all;
    TRY(cudaMallocAsync(&d_fr, sizeof(int2), st));
    TRY(cudaMemcpyAsync(d_fr, hfront.data(), sizeof(int2), cudaMemcpyHostToDevice, st));
    for (int l = 0; l <= depth && nf > 0; ++l) {
      int32_t *d_occ = nullptr;
      TRY(cudaMallocAsync(&d_occ, sizeof(int32_t) * 2 * (nf + 1), st));
      d_oc = d_occ;
      d_cc = d_occ + (nf + 1);
      TRY(cudaMallocAsync(&d_kind, nf, st));
      TRY(cudaMemsetAsync(d_occ, 0, sizeof(int32_t) * 2 * (nf + 1), st));
      k_bt_classify<<<nblk(nf, 256), 256, 0, st>>>(d_fr, nf, l, depth, d, T.box, eta, d_oc, d_cc,
                                                    d_kind);
      k_scan_excl<<<1, 1024, 0, st>>>(d_oc, nf + 1);
      k_scan_excl<<<1, 1024, 0, st>>>(d_cc, nf + 1);
      int32_t tot[2];
      TRY(cudaMemcpyAsync(&tot[0], d_oc + nf, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      TRY(cudaMemcpyAsync(&tot[1], d_cc + nf, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
      TRY(cudaStreamSynchronize(st));
      TRY(cudaMallocAsync(&d_blocks, sizeof(int4) * (tot[0] > 0 ? tot[0] : 1), st));
      TRY(cudaMallocAsync(&d_next, sizeof(int2) * (tot[1] > 0 ? tot[1] : 1), st));
      k_bt_emit<<<nblk(nf, 256), 256, 0, st>>>(d_fr, nf, l, d_kind, d_oc, d_cc, d_blocks, 0, d_next);
      TRY(cudaGetLastError());
      if (tot[0] > 0) {
        size_t old = all.size();
        all.resize(old + tot[0]);
        TRY(cudaMemcpyAsync(all.data() + old, d_blocks, sizeof(int4) * tot[0],
                            cudaMemcpyDeviceToHost, st));
      }
      TRY(cudaStreamSynchronize(st));
      cudaFreeAsync(d_occ, st);
      cudaFreeAsync(d_kind, st);
      cudaFreeAsync(d_blocks, st);
      cudaFreeAsync(d_fr, st);
      d_fr = d_next;
      d_next = nullptr;
      nf = tot[1];
    }
    cudaFreeAsync(d_fr, st);
    blocks_out.swap(all);
  }
done:
#undef TRY
  cudaFreeAsync(d_beg, st); cudaFreeAsync(d_end, st); cudaFreeAsync(d_cop, st);
  cudaFreeAsync(d_val, st); cudaFreeAsync(d_val2, st); cudaFreeAsync(d_perm2, st);
  cudaFreeAsync(d_key, st); cudaFreeAsync(d_key2, st); cudaFreeAsync(d_xyz2, st);
  cudaFreeAsync(d_hist, st); cudaFreeAsync(d_bad, st);
  cudaStreamSynchronize(st);
  return err;
}

}  // namespace hmle
