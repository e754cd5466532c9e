// Cluster tree / block tree construction on the device (tree.cu).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

namespace hmle {

struct DeviceTree {
  double *xyz = nullptr;   // coordinates in cluster order, SoA (3 x n)
  int32_t *perm = nullptr; // perm[k] = caller index of cluster position k
  double *box = nullptr;   // per heap cluster: lo[3], hi[3]
};

// rows_dev: n x d row-major coordinates on the device.  cl_beg / cl_end:
// heap-indexed cluster ranges (levels 0..depth).  On success fills T and
// the block list (level, i, j, kind) with kind 0 = dense leaf, 1 = admissible.
std::string tree_build_device(cudaStream_t st, const double *rows_dev, int64_t n, int d,
                              int depth, const std::vector<int32_t> &cl_beg,
                              const std::vector<int32_t> &cl_end, double eta,
                              DeviceTree &T, std::vector<int4> &blocks_out);

}  // namespace hmle
