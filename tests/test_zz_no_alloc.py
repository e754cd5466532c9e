"""The no-allocation Matern entry point (hmle_matern_eval_noalloc).

Some callers cannot allocate device memory while they call this library: a
CUDA graph being captured does not allow cudaMalloc, and some hosts give the
library a fixed device-memory budget.  For them the Matern-table evaluation
has a variant whose scratch (one Chebyshev table per nu) is a static device
array, and whose inputs and outputs are the caller's device buffers.  This
file checks it, through the C ABI, against the allocating entry point
(hmle_matern_eval) on two calls in a row, which share and overwrite that
static array.  It is collected last, so that a run stopping at the first
failure has run every other test before it.
"""
import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _call(lib, ctx, nus, xd, m, outd):
    arr = (C.c_double * len(nus))(*nus)
    return lib.hmle_matern_eval_noalloc(ctx._h, arr, len(nus), C.c_void_p(xd.data_ptr()), m,
                                        C.c_void_p(outd.data_ptr()))


def test_noalloc_matches_allocating_entry_point(hmle_lib):
    import torch
    from paper_2104_07146_gb300 import hmle
    ctx = hmle.Context()
    x = np.concatenate([[0.0, 1e-6], np.logspace(-4, 3.05, 997)])
    m = x.size
    xd = torch.from_numpy(x).cuda()
    runs = [[0.5, 1.5, 2.5, 0.3, 0.8], [2.2, 0.7, 1.0]]   # two calls, the second overwrites
    for nus in runs:
        outd = torch.full((len(nus) * m,), float("nan"), dtype=torch.float64, device="cuda")
        assert _call(hmle_lib, ctx, nus, xd, m, outd) == 0
        torch.cuda.synchronize()
        out = outd.cpu().numpy()
        for j, nu in enumerate(nus):
            ref = ctx.matern(nu, x)                       # allocating entry point
            assert np.max(np.abs(out[j * m:(j + 1) * m] - ref)) <= 1e-13


def test_noalloc_rejects_what_it_cannot_hold(hmle_lib):
    import torch
    from paper_2104_07146_gb300 import hmle
    ctx = hmle.Context()
    xd = torch.linspace(0, 1, 10, dtype=torch.float64, device="cuda")
    outd = torch.empty(17 * 10, dtype=torch.float64, device="cuda")
    assert _call(hmle_lib, ctx, [0.5] * 17, xd, 10, outd) == 1     # more tables than the static array
    xh = torch.linspace(0, 1, 10, dtype=torch.float64)              # host input: nothing is staged
    assert _call(hmle_lib, ctx, [0.5], xh, 10, outd) == 1
