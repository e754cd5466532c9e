// Per-kernel algorithmic FP64 flop tally of one evaluation (tally.cpp).
#pragma once

#include <stdint.h>

#include <cmath>
#include <vector>

#include "hmle_internal.h"

namespace hmle {

// kind: index into kKernelNames (kernels.cuh).  rc / rl: ACA ranks of C and
// ranks of L per block; kept: kept columns per low-rank target;
// jacobi_flops: the device count of the Jacobi sweeps of that evaluation.
double tally_flops(const Plan &P, int kind, const std::vector<int32_t> &rc,
                   const std::vector<int32_t> &rl, const std::vector<int32_t> &kept, int osamp,
                   double jacobi_flops);

}  // namespace hmle
