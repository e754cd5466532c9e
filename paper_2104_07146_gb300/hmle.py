"""ctypes binding of libhmle.so (include/hmle.h).  Argument marshalling only:
every numerical step runs in the library's CUDA kernels.  Arrays may be numpy
arrays (host) or torch tensors (host or CUDA); they are passed by pointer.

If the shared library is missing it is built with nvcc (``build.py``); if that
is impossible the import of ``lib()`` raises -- there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import sys

import numpy as np

from . import build as _build

HMLE_OK = 0
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "NOT_SPD", 3: "OOM", 4: "CUDA", 5: "RANK_OVERFLOW",
          6: "TIMEOUT", 7: "NOT_CONVERGED", 8: "NOT_IMPLEMENTED"}


class HmleError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__("%s: %s" % (STATUS.get(status, status), msg))
        self.status = status


HMLE_FP64 = 0
HMLE_MIXED_FP32 = 1
HMLE_MIXED_BF16 = 2


class Opts(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("eta", C.c_double), ("aca_eps", C.c_double),
                ("max_rank", C.c_int32), ("oversample", C.c_int32), ("precision", C.c_int32),
                ("seed", C.c_uint64), ("leaf_lowrank", C.c_int32), ("pcg_tol", C.c_double),
                ("pcg_max_iter", C.c_int32), ("fixed_rank", C.c_int32), ("batch_size", C.c_int32)]


class FitOpts(C.Structure):
    _fields_ = [("ftol", C.c_double), ("xtol", C.c_double), ("max_iter", C.c_int32),
                ("step", C.c_double * 4)]


class Theta(C.Structure):
    _fields_ = [("ell", C.c_double), ("nu", C.c_double), ("sigma2", C.c_double),
                ("tau2", C.c_double)]


class TreeInfo(C.Structure):
    _fields_ = [("n", C.c_int64), ("d", C.c_int32), ("depth", C.c_int32),
                ("n_leaves", C.c_int32), ("n_dense", C.c_int32), ("n_lowrank", C.c_int32),
                ("dense_words", C.c_int64), ("lowrank_words", C.c_int64),
                ("device_bytes", C.c_int64)]


class Task(C.Structure):
    _fields_ = [("tree", C.c_void_p), ("theta", Theta), ("Z", C.c_void_p)]


class RetryInfo(C.Structure):
    _fields_ = [("retries", C.c_int32), ("max_rank", C.c_int32), ("precision", C.c_int32),
                ("aca_eps", C.c_double)]


class TuneResult(C.Structure):
    _fields_ = [("leaf_size", C.c_int32), ("concurrency", C.c_int32), ("evals_per_s", C.c_double),
                ("trials", C.c_int32), ("batch_size", C.c_int32)]


class EvalInfo(C.Structure):
    _fields_ = [("logdet", C.c_double), ("quad", C.c_double), ("loglik", C.c_double),
                ("max_rank_c", C.c_int32), ("max_rank_l", C.c_int32),
                ("mean_rank_l", C.c_double), ("status", C.c_int32),
                ("kernel_launches", C.c_int64), ("pcg_iters", C.c_int32),
                ("pcg_relres", C.c_double), ("flops", C.c_double)]


_LIB = None
P = C.c_void_p
OBJECTIVE = C.CFUNCTYPE(C.c_double, C.POINTER(C.c_double), C.c_int32, C.c_void_p)


def lib():
    """Load libhmle.so (building it with nvcc when missing or stale)."""
    global _LIB
    if _LIB is None:
        path = _build.build()
        L = C.CDLL(path)
        sigs = {
            "hmle_opts_default": ([P], C.c_int),
            "hmle_fit_opts_default": ([P], C.c_int),
            "hmle_ctx_create": ([P, P], C.c_int),
            "hmle_ctx_destroy": ([P], None),
            "hmle_last_error": ([P], C.c_char_p),
            "hmle_build_tree": ([P, P, C.c_int64, C.c_int32, P, P], C.c_int),
            "hmle_tree_destroy": ([P], None),
            "hmle_tree_get_info": ([P, P], C.c_int),
            "hmle_tree_permutation": ([P, P], C.c_int),
            "hmle_assemble": ([P, P, P, P], C.c_int),
            "hmle_hmatrix_destroy": ([P], None),
            "hmle_hmatrix_matvec": ([P, P, P, P], C.c_int),
            "hmle_factor": ([P, P, P, P], C.c_int),
            "hmle_factor_destroy": ([P], None),
            "hmle_loglik": ([P, P, P, P, P, P], C.c_int),
            "hmle_loglik_eval": ([P, P, P, P, P, P], C.c_int),
            "hmle_fit": ([P, P, P, P, P, P, P, P, P], C.c_int),
            "hmle_matern_eval": ([P, C.c_double, P, C.c_int64, P], C.c_int),
            "hmle_profile_select": ([P, C.c_char_p], C.c_int),
            "hmle_simulate": ([P, P, P, P, P], C.c_int),
            "hmle_loglik_batch": ([P, P, P, C.c_int32, P, C.c_int32, P, P], C.c_int),
            "hmle_solve": ([P, P, P, P], C.c_int),
            "hmle_predict": ([P, P, P, P, C.c_int64, P], C.c_int),
            "hmle_cross_matvec": ([P, P, P, P, C.c_int64, C.c_int32, P, P], C.c_int),
            "hmle_fit_profiled": ([P, P, P, P, P, P, P, P, P], C.c_int),
            "hmle_loglik_multi": ([P, P, C.c_int32, C.c_int32, P, P], C.c_int),
            "hmle_loglik_multi_retry": ([P, P, C.c_int32, C.c_int32, C.c_int32, P, P, P], C.c_int),
            "hmle_prediction_errors": ([P, P, P, P, C.c_int64, P, P, P], C.c_int),
            "hmle_theta_to_x": ([P, P], C.c_int),
            "hmle_selftest_barrier": ([P, C.c_int32, P], C.c_int),
            "hmle_selftest_tc_gemm": ([P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32,
                                       C.c_int32, C.c_int32, P, P, P], C.c_int),
            "hmle_x_to_theta": ([P, P], C.c_int),
            "hmle_features": ([P, P, C.c_int64, C.c_int32, P, P], C.c_int),
            "hmle_mlp_nparams": ([], C.c_int32),
            "hmle_mlp_create": ([P, C.c_uint64, P], C.c_int),
            "hmle_mlp_destroy": ([P], None),
            "hmle_mlp_set": ([P, P, P, P, P], C.c_int),
            "hmle_mlp_get": ([P, P, P, P, P], C.c_int),
            "hmle_mlp_forward": ([P, P, P, C.c_int32, P], C.c_int),
            "hmle_mlp_grad": ([P, P, P, P, C.c_int32, P, P], C.c_int),
            "hmle_mlp_adam_step": ([P, P, P, C.c_float], C.c_int),
            "hmle_mlp_train": ([P, P, P, P, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_uint64,
                                P, P], C.c_int),
            "hmle_tree_set_batch_size": ([P, C.c_int32], C.c_int),
            "hmle_autotune": ([P, P, C.c_int64, C.c_int32, P, P, P, C.c_int32, P, P, C.c_int32, P],
                              C.c_int),
            "hmle_matern_eval_noalloc": ([P, P, C.c_int32, P, C.c_int64, P], C.c_int),
            "hmle_profile_read": ([P, P, P, P], C.c_int),
            "hmle_phase_work": ([P, P, P, P], C.c_int),
            "hmle_plan_build": ([C.c_int64, C.c_int32, C.c_int32, P, C.c_int32, C.c_int32,
                                 C.c_int32, P], C.c_int),
            "hmle_plan_destroy": ([P], None),
            "hmle_nelder_mead": ([C.c_int32, OBJECTIVE, P, P, P, P, P, P, P, P], C.c_int),
            "hmle_plan_list": ([P, C.c_int32, P, C.c_int64, P, P], C.c_int),
        }
        for name, (argt, rest) in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = argt
            fn.restype = rest
        _LIB = L
    return _LIB


def exported_symbols():
    """Names declared in include/hmle.h (for the ABI check)."""
    return ["hmle_opts_default", "hmle_fit_opts_default", "hmle_ctx_create", "hmle_ctx_destroy",
            "hmle_last_error", "hmle_build_tree", "hmle_tree_destroy", "hmle_tree_get_info",
            "hmle_tree_permutation", "hmle_assemble", "hmle_hmatrix_destroy",
            "hmle_hmatrix_matvec", "hmle_factor", "hmle_factor_destroy", "hmle_loglik",
            "hmle_loglik_eval", "hmle_fit", "hmle_matern_eval", "hmle_profile_select",
            "hmle_profile_read", "hmle_phase_work", "hmle_simulate", "hmle_loglik_batch", "hmle_solve", "hmle_predict", "hmle_fit_profiled", "hmle_cross_matvec", "hmle_loglik_multi", "hmle_loglik_multi_retry", "hmle_prediction_errors", "hmle_autotune", "hmle_tree_set_batch_size",
            "hmle_theta_to_x", "hmle_x_to_theta", "hmle_selftest_barrier", "hmle_selftest_tc_gemm", "hmle_features", "hmle_mlp_nparams",
            "hmle_mlp_create", "hmle_mlp_destroy", "hmle_mlp_set", "hmle_mlp_get",
            "hmle_mlp_forward", "hmle_mlp_grad", "hmle_mlp_adam_step", "hmle_mlp_train",
            "hmle_matern_eval_noalloc", "hmle_plan_build", "hmle_plan_destroy",
            "hmle_plan_list", "hmle_nelder_mead"]


def _ptr(a):
    """(pointer, keepalive) for a numpy array or torch tensor of float64/int32."""
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            a = a.contiguous()
        return C.c_void_p(a.data_ptr()), a
    a = np.ascontiguousarray(a)
    return C.c_void_p(a.ctypes.data), a


class Context:
    """An hmle_ctx on the current CUDA device.  stream: a torch.cuda.Stream,
    a raw cudaStream_t integer, or None for a library-owned stream."""

    def __init__(self, stream=None):
        L = lib()
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        self._h = P()
        st = L.hmle_ctx_create(C.byref(self._h), P(stream) if stream else None)
        if st != HMLE_OK:
            raise HmleError(st, "hmle_ctx_create")

    def last_error(self) -> str:
        msg = lib().hmle_last_error(self._h)
        return msg.decode() if msg else ""

    def check(self, st, what=""):
        if st != HMLE_OK:
            msg = lib().hmle_last_error(self._h)
            raise HmleError(st, (what + ": " if what else "") + (msg.decode() if msg else ""))

    @staticmethod
    def _tasks(tasks):
        tasks = list(tasks)
        keep = []
        arr = (Task * max(len(tasks), 1))()
        for i, (tree, th, Z) in enumerate(tasks):
            p, k = _ptr(Z)
            keep.append(k)
            arr[i].tree = tree._h
            arr[i].theta = _theta(th)
            arr[i].Z = p.value
        return arr, len(tasks), keep

    def loglik_multi(self, tasks, concurrency=8):
        """Evaluations over several trees at once: tasks = [(tree, theta, Z), ...].
        Returns (L array, status array)."""
        arr, m, keep = self._tasks(tasks)
        ll = np.empty(m, dtype=np.float64)
        stt = np.empty(m, dtype=np.int32)
        self.check(lib().hmle_loglik_multi(self._h, arr, m, int(concurrency), P(ll.ctypes.data),
                                           P(stt.ctypes.data)), "hmle_loglik_multi")
        return ll, stt

    def loglik_multi_retry(self, tasks, concurrency=8, max_retries=3):
        """loglik_multi with failed tasks retried on derived trees
        (hmle_loglik_multi_retry).  Returns (L array, status array, list of
        per-task dicts: retries, max_rank, precision, aca_eps)."""
        arr, m, keep = self._tasks(tasks)
        ll = np.empty(m, dtype=np.float64)
        stt = np.empty(m, dtype=np.int32)
        info = (RetryInfo * max(m, 1))()
        self.check(lib().hmle_loglik_multi_retry(self._h, arr, m, int(concurrency), int(max_retries),
                                                 P(ll.ctypes.data), P(stt.ctypes.data), info),
                   "hmle_loglik_multi_retry")
        return ll, stt, [{"retries": int(info[i].retries), "max_rank": int(info[i].max_rank),
                          "precision": int(info[i].precision), "aca_eps": float(info[i].aca_eps)}
                         for i in range(m)]

    def autotune(self, locs, theta, Z, max_concurrency=16, **opts):
        """hmle_autotune: returns (best dict, list of trial dicts)."""
        locs = np.ascontiguousarray(locs, dtype=np.float64)
        n, d = locs.shape
        o = default_opts(**opts)
        best = TuneResult()
        trials = (TuneResult * 64)()
        nt = C.c_int32()
        p, keep = _ptr(Z)
        self.check(lib().hmle_autotune(self._h, P(locs.ctypes.data), n, d, C.byref(o),
                                       C.byref(_theta(theta)), p, int(max_concurrency),
                                       C.byref(best), trials, 64, C.byref(nt)), "hmle_autotune")
        conv = lambda r: {"leaf_size": r.leaf_size, "concurrency": r.concurrency,
                          "batch_size": r.batch_size, "evals_per_s": r.evals_per_s}
        return conv(best), [conv(trials[i]) for i in range(min(nt.value, 64))]

    def close(self):
        if self._h:
            lib().hmle_ctx_destroy(self._h)
            self._h = P()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass

    def matern(self, nu: float, x) -> np.ndarray:
        """M_nu(x) as the device evaluates it (host float64 arrays)."""
        x = np.ascontiguousarray(x, dtype=np.float64)
        out = np.empty_like(x)
        self.check(lib().hmle_matern_eval(self._h, float(nu), P(x.ctypes.data), x.size,
                                          P(out.ctypes.data)), "hmle_matern_eval")
        return out

    def tc_gemm(self, A, B, nslices: int, a_kfast: bool = True, b_kfast: bool = True,
                copies: int = 1) -> np.ndarray:
        """C = A B by the tensor-core tile product with nslices BF16 slices
        per operand (hmle_selftest_tc_gemm); returns copies x M x N."""
        A = np.ascontiguousarray(A, dtype=np.float64)
        B = np.ascontiguousarray(B, dtype=np.float64)
        M, K = A.shape
        K2, N = B.shape
        assert K == K2
        out = np.empty((copies, N, M), dtype=np.float64)
        self.check(lib().hmle_selftest_tc_gemm(self._h, nslices, int(a_kfast), int(b_kfast), copies, M, N, K,
                                               P(A.ctypes.data), P(B.ctypes.data), P(out.ctypes.data)),
                   "hmle_selftest_tc_gemm")
        return out.transpose(0, 2, 1)


class Profiler:
    """Per-kernel CUDA-event timing and flop tally (hmle_profile_*)."""

    def __init__(self, ctx: Context, kernel: str):
        self.ctx = ctx
        self.kernel = kernel
        self.enabled = False

    def enable(self, on: bool):
        name = self.kernel.encode() if on else None
        self.ctx.check(lib().hmle_profile_select(self.ctx._h, name), "hmle_profile_select")
        self.enabled = on

    def reset(self):
        if self.enabled:
            self.enable(True)

    def read(self):
        ms, n, fl = C.c_double(), C.c_int64(), C.c_double()
        self.ctx.check(lib().hmle_profile_read(self.ctx._h, C.byref(ms), C.byref(n), C.byref(fl)),
                       "hmle_profile_read")
        return {"name": self.kernel, "ms": ms.value, "launches": n.value, "flops": fl.value}


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().hmle_opts_default(C.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def _theta(theta) -> Theta:
    if isinstance(theta, Theta):
        return theta
    ell, nu, s2, t2 = (float(v) for v in theta)
    return Theta(ell, nu, s2, t2)


class Tree:
    """hmle_build_tree: cluster tree, block tree and factorisation schedule."""

    def __init__(self, ctx: Context, locs, opts: Opts | None = None, **kw):
        self.ctx = ctx
        if opts is None:
            opts = default_opts(**kw)
        self.opts = opts
        if hasattr(locs, "shape"):
            n, d = int(locs.shape[0]), int(locs.shape[1])
        else:
            locs = np.asarray(locs, dtype=np.float64)
            n, d = locs.shape
        if not hasattr(locs, "data_ptr"):
            locs = np.ascontiguousarray(locs, dtype=np.float64)
        p, keep = _ptr(locs)
        self._h = P()
        ctx.check(lib().hmle_build_tree(ctx._h, p, n, d, C.byref(opts), C.byref(self._h)),
                  "hmle_build_tree")
        self.n, self.d = n, d

    def info(self) -> TreeInfo:
        i = TreeInfo()
        self.ctx.check(lib().hmle_tree_get_info(self._h, C.byref(i)), "hmle_tree_get_info")
        return i

    def permutation(self) -> np.ndarray:
        perm = np.empty(self.n, dtype=np.int32)
        self.ctx.check(lib().hmle_tree_permutation(self._h, P(perm.ctypes.data)),
                       "hmle_tree_permutation")
        return perm

    def loglik(self, theta, Z):
        """One evaluation of Eq. 1: returns (L, EvalInfo)."""
        p, keep = _ptr(Z)
        ll = C.c_double()
        info = EvalInfo()
        st = lib().hmle_loglik_eval(self.ctx._h, self._h, C.byref(_theta(theta)), p,
                                    C.byref(ll), C.byref(info))
        self.ctx.check(st, "hmle_loglik_eval")
        return ll.value, info

    def loglik_batch(self, thetas, Z, concurrency=8):
        """m evaluations of Eq. 1 run concurrently: returns (L array, status array)."""
        thetas = list(thetas)
        m = len(thetas)
        arr = (Theta * max(m, 1))(*[_theta(t) for t in thetas])
        ll = np.empty(m, dtype=np.float64)
        stt = np.empty(m, dtype=np.int32)
        p, keep = _ptr(Z)
        st = lib().hmle_loglik_batch(self.ctx._h, self._h, arr, m, p, int(concurrency),
                                     P(ll.ctypes.data), P(stt.ctypes.data))
        self.ctx.check(st, "hmle_loglik_batch")
        return ll, stt

    def simulate(self, theta, xi) -> np.ndarray:
        """Z = P^T L~ P xi: a sample of the field with covariance C~(theta)."""
        xi = np.ascontiguousarray(xi, dtype=np.float64)
        Z = np.empty_like(xi)
        self.ctx.check(lib().hmle_simulate(self.ctx._h, self._h, C.byref(_theta(theta)),
                                           P(xi.ctypes.data), P(Z.ctypes.data)), "hmle_simulate")
        return Z

    def cross_matvec(self, theta, locs2, x, trans=False) -> np.ndarray:
        """C21 x (trans=False; x of length n) or C12 x (trans=True; x of length m)
        between this tree's points and the m x d locations locs2."""
        L2 = np.ascontiguousarray(locs2, dtype=np.float64)
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty(self.n if trans else L2.shape[0])
        self.ctx.check(lib().hmle_cross_matvec(self.ctx._h, self._h, C.byref(_theta(theta)),
                                               P(L2.ctypes.data), L2.shape[0], int(trans),
                                               P(x.ctypes.data), P(y.ctypes.data)),
                       "hmle_cross_matvec")
        return y

    def assemble(self, theta) -> "HMatrix":
        return HMatrix(self, theta)

    def fit(self, Z, theta0, ftol=1e-4, xtol=1e-4, max_iter=400, step=None, profiled=False):
        """Nelder-Mead MLE: returns (theta_hat tuple, L_hat, iterations, evaluations, status).
        profiled=True: sigma2 profiled out, a 3-coordinate search (hmle_fit_profiled)."""
        fo = FitOpts()
        lib().hmle_fit_opts_default(C.byref(fo))
        fo.ftol, fo.xtol, fo.max_iter = ftol, xtol, max_iter
        if step is not None:
            for i in range(4):
                fo.step[i] = float(step[i])
        p, keep = _ptr(Z)
        th = Theta()
        ll = C.c_double()
        it = C.c_int32()
        nev = C.c_int32()
        fn = lib().hmle_fit_profiled if profiled else lib().hmle_fit
        st = fn(self.ctx._h, self._h, p, C.byref(_theta(theta0)), C.byref(fo),
                C.byref(th), C.byref(ll), C.byref(it), C.byref(nev))
        if st not in (HMLE_OK, 7):
            self.ctx.check(st, "hmle_fit")
        return (th.ell, th.nu, th.sigma2, th.tau2), ll.value, it.value, nev.value, st

    def close(self):
        if self._h:
            lib().hmle_tree_destroy(self._h)
            self._h = P()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


def nelder_mead(f, x0, step=None, ftol=1e-4, xtol=1e-4, max_iter=400):
    """hmle_nelder_mead: minimise f(x) (x a numpy array) with the optimiser
    of hmle_fit.  Returns (x_best, f_best, iterations, evaluations, status)."""
    x0 = np.ascontiguousarray(x0, dtype=np.float64)
    dim = x0.size
    st = None if step is None else np.ascontiguousarray(
        np.broadcast_to(np.asarray(step, dtype=np.float64), (dim,)))
    fo = FitOpts()
    lib().hmle_fit_opts_default(C.byref(fo))
    fo.ftol, fo.xtol, fo.max_iter = ftol, xtol, max_iter

    def cb(x, d, user):
        return float(f(np.ctypeslib.as_array(x, shape=(d,)).copy()))
    fn = OBJECTIVE(cb)
    xb = np.zeros(dim)
    fb = C.c_double()
    it, nev = C.c_int32(), C.c_int32()
    status = lib().hmle_nelder_mead(dim, fn, None, P(x0.ctypes.data),
                                    None if st is None else P(st.ctypes.data), C.byref(fo),
                                    P(xb.ctypes.data), C.byref(fb), C.byref(it), C.byref(nev))
    if status not in (HMLE_OK, 7):
        raise HmleError(status, "hmle_nelder_mead")
    return xb, fb.value, it.value, nev.value, status


PLAN_LISTS = ["scalars", "blocks", "steps", "lrt", "aent", "bent", "lrpairs", "dns", "dpairs",
              "panels", "wpan", "hts", "urows", "uents", "grams", "gchunks", "greds", "arow",
              "brow", "arow_ent", "brow_ent", "apair", "bpair", "hts_rhs", "urows_rhs",
              "uents_rhs", "ht_rhs0", "ur_rhs0", "bh_blocks", "bh0", "bupd", "bents", "bupd0",
              "mv_row0", "mv_blocks", "mvt_row0", "mvt_blocks"]


class Plan:
    """hmle_plan_build: the schedule of the leaf sweep for a given block
    partition, built on the host (no device).  blocks: (level, i, j, kind)
    rows; list(name) returns one of PLAN_LISTS as an int64 array of records
    (fields as in include/hmle.h)."""

    def __init__(self, n, d, leaf_size, blocks, max_rank=32, oversample=8):
        b = np.ascontiguousarray(blocks, dtype=np.int32).reshape(-1, 4)
        self._h = P()
        st = lib().hmle_plan_build(int(n), int(d), int(leaf_size), P(b.ctypes.data), b.shape[0],
                                   int(max_rank), int(oversample), C.byref(self._h))
        if st != HMLE_OK:
            raise HmleError(st, "hmle_plan_build")

    def list(self, name) -> np.ndarray:
        which = PLAN_LISTS.index(name)
        nrec, width = C.c_int64(), C.c_int32()
        st = lib().hmle_plan_list(self._h, which, None, 0, C.byref(nrec), C.byref(width))
        if st != HMLE_OK:
            raise HmleError(st, "hmle_plan_list")
        out = np.zeros((nrec.value, width.value), dtype=np.int64)
        if out.size:
            st = lib().hmle_plan_list(self._h, which, P(out.ctypes.data), out.size, None, None)
            if st != HMLE_OK:
                raise HmleError(st, "hmle_plan_list")
        return out

    def close(self):
        if self._h:
            lib().hmle_plan_destroy(self._h)
            self._h = P()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class HMatrix:
    """hmle_assemble: C~(theta) held as an H-matrix on the device."""

    def __init__(self, tree: Tree, theta):
        self.tree = tree
        self._h = P()
        tree.ctx.check(lib().hmle_assemble(tree.ctx._h, tree._h, C.byref(_theta(theta)),
                                           C.byref(self._h)), "hmle_assemble")

    def matvec(self, x) -> np.ndarray:
        x = np.ascontiguousarray(x, dtype=np.float64)
        y = np.empty_like(x)
        self.tree.ctx.check(lib().hmle_hmatrix_matvec(self.tree.ctx._h, self._h, P(x.ctypes.data),
                                                      P(y.ctypes.data)), "hmle_hmatrix_matvec")
        return y

    def factor(self, Z=None) -> "Factor":
        return Factor(self, Z)

    def close(self):
        if self._h:
            lib().hmle_hmatrix_destroy(self._h)
            self._h = P()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass


class Factor:
    """hmle_factor: the H-Cholesky factor (with the forward solve of Z fused)."""

    def __init__(self, hm: HMatrix, Z=None):
        self.hm = hm
        self._h = P()
        self._Z = Z
        p, keep = _ptr(Z) if Z is not None else (None, None)
        ctx = hm.tree.ctx
        ctx.check(lib().hmle_factor(ctx._h, hm._h, p, C.byref(self._h)), "hmle_factor")

    def loglik(self, Z=None):
        """(L, log|C~|, Z^T C~^{-1} Z); Z = None uses the solve fused into the factor."""
        p, keep = _ptr(Z) if Z is not None else (None, None)
        ll, ld, q = C.c_double(), C.c_double(), C.c_double()
        ctx = self.hm.tree.ctx
        ctx.check(lib().hmle_loglik(ctx._h, self._h, p, C.byref(ll), C.byref(ld), C.byref(q)),
                  "hmle_loglik")
        return ll.value, ld.value, q.value

    def solve(self, Z) -> np.ndarray:
        """X = C~^{-1} Z (forward and backward sweeps through the factor)."""
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        X = np.empty_like(Z)
        ctx = self.hm.tree.ctx
        ctx.check(lib().hmle_solve(ctx._h, self._h, P(Z.ctypes.data), P(X.ctypes.data)), "hmle_solve")
        return X

    def phase_work(self):
        """(assembly FP64 flops, bytes of the factor read by one hmle_solve)."""
        fa, sb = C.c_double(), C.c_double()
        ctx = self.hm.tree.ctx
        ctx.check(lib().hmle_phase_work(ctx._h, self._h, C.byref(fa), C.byref(sb)),
                  "hmle_phase_work")
        return fa.value, sb.value

    def predict(self, Z, locs2) -> np.ndarray:
        """Kriging prediction (Eq. 4) at the m x d locations locs2."""
        Z = np.ascontiguousarray(Z, dtype=np.float64)
        L2 = np.ascontiguousarray(locs2, dtype=np.float64)
        out = np.empty(L2.shape[0])
        ctx = self.hm.tree.ctx
        ctx.check(lib().hmle_predict(ctx._h, self._h, P(Z.ctypes.data), P(L2.ctypes.data),
                                     L2.shape[0], P(out.ctypes.data)), "hmle_predict")
        return out

    def prediction_errors(self, approx: "Factor", locs2):
        """hmle_prediction_errors with this factor as the true model and
        `approx` as the approximated one: (MLOE, MMOM, per-location array
        m x 3 of E_t[(Z_t - Z)^2], E_a[(Z_a - Z)^2], E_t[(Z_a - Z)^2])."""
        L2 = np.ascontiguousarray(locs2, dtype=np.float64)
        m = L2.shape[0]
        per = np.empty((m, 3))
        a, b = C.c_double(), C.c_double()
        ctx = self.hm.tree.ctx
        ctx.check(lib().hmle_prediction_errors(ctx._h, self._h, approx._h, P(L2.ctypes.data), m,
                                               C.byref(a), C.byref(b), P(per.ctypes.data)),
                  "hmle_prediction_errors")
        return a.value, b.value, per

    def close(self):
        if self._h:
            lib().hmle_factor_destroy(self._h)
            self._h = P()

    def __del__(self):
        if sys.is_finalizing():
            return
        try:
            self.close()
        except Exception:
            pass
