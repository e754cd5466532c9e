"""The C-ABI library builds, loads, and exports every symbol the header
declares (no compute call: runs without a GPU)."""
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hmle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hmle_[a-z_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ["hmle_build_tree", "hmle_assemble", "hmle_factor", "hmle_loglik", "hmle_fit"]:
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2104_07146_gb300 import hmle
    L = hmle.lib()
    for name in _declared():
        assert hasattr(L, name), name
    assert sorted(hmle.exported_symbols()) == _declared()


# --- host-only entry points, called without a GPU -----------------------------

import ctypes as C
import math

import numpy as np
import pytest

import oracle
from oracle import learned_start as oracle_ls


def _lib():
    from paper_2104_07146_gb300 import hmle
    return hmle, hmle.lib()


def test_theta_transform_matches_the_oracle():
    # Sec. 5 positivity transform on the host side of the library against the
    # oracle's restatement, over the prior box and beyond it
    hmle, L = _lib()
    rng = np.random.default_rng(5)
    for _ in range(200):
        th = (float(np.exp(rng.uniform(-6, 3))), float(rng.uniform(0.05, 20.0)),
              float(np.exp(rng.uniform(-5, 5))), float(np.exp(rng.uniform(-12, 2))))
        x = (C.c_double * 4)()
        assert L.hmle_theta_to_x(C.byref(hmle._theta(th)), x) == 0
        ref = oracle.untransform(th)
        np.testing.assert_allclose(list(x), ref, rtol=1e-13, atol=1e-13)
        back = hmle.Theta()
        assert L.hmle_x_to_theta(x, C.byref(back)) == 0
        np.testing.assert_allclose([back.ell, back.nu, back.sigma2, back.tau2],
                                   oracle.transform(ref), rtol=1e-12)
        np.testing.assert_allclose([back.ell, back.nu, back.sigma2, back.tau2], th, rtol=1e-12)


def test_theta_transform_golden_start_point():
    # the paper's initial guess in transformed coordinates (Sec. 5, Test 1a),
    # with theta written out by hand in tests/golden/transform_start.json
    import json
    hmle, L = _lib()
    g = json.load(open(os.path.join(ROOT, "tests", "golden", "transform_start.json")))
    th = hmle.Theta()
    assert L.hmle_x_to_theta((C.c_double * 4)(*g["x0"]), C.byref(th)) == 0
    assert abs(math.sqrt(th.sigma2) - g["sigma"]) <= 1e-15
    assert abs(th.ell - g["ell"]) <= 1e-15
    assert abs(th.nu - g["nu"]) <= 1e-15
    assert abs(math.sqrt(th.tau2) - g["tau"]) <= 1e-20
    x = (C.c_double * 4)()
    assert L.hmle_theta_to_x(C.byref(th), x) == 0
    np.testing.assert_allclose(list(x), g["x0"], rtol=1e-13)


@pytest.mark.parametrize("th", [(0.0, 1.0, 1.0, 0.1), (-1.0, 1.0, 1.0, 0.1), (0.1, 0.0, 1.0, 0.1),
                                (0.1, 20.5, 1.0, 0.1), (0.1, 1.0, 0.0, 0.1), (0.1, 1.0, 1.0, 0.0),
                                (float("nan"), 1.0, 1.0, 0.1), (0.1, 1.0, float("inf"), 0.1)])
def test_theta_to_x_rejects_out_of_range(th):
    # sigma2 = 0 or tau2 = 0 has no transformed coordinate (log 0)
    hmle, L = _lib()
    x = (C.c_double * 4)()
    assert L.hmle_theta_to_x(C.byref(hmle._theta(th)), x) == 1


@pytest.mark.parametrize("x", [(float("nan"), 0, 0, 0), (0, float("inf"), 0, 0),
                               (0, 0, -20.0, 0)])
def test_x_to_theta_rejects_non_finite_and_out_of_range(x):
    # x[2] = -20 gives nu = 1.2^20 = 38 > 20, outside the admissible range
    hmle, L = _lib()
    th = hmle.Theta()
    assert L.hmle_x_to_theta((C.c_double * 4)(*x), C.byref(th)) == 1


def test_opts_default_and_null_arguments():
    hmle, L = _lib()
    o = hmle.Opts()
    assert L.hmle_opts_default(C.byref(o)) == 0
    assert (o.leaf_size, o.eta, o.aca_eps, o.max_rank, o.oversample, o.precision) == \
        (64, 2.0, 1e-8, 32, 8, 0)
    assert L.hmle_opts_default(None) == 1
    assert L.hmle_theta_to_x(None, (C.c_double * 4)()) == 1
    assert L.hmle_x_to_theta(None, None) == 1


def test_mlp_parameter_count_matches_the_oracle():
    # 35-64-64-8 perceptron: weights and biases of three layers
    _, L = _lib()
    assert L.hmle_mlp_nparams() == oracle_ls.NPARAMS == 35 * 256 + 256 + 2 * (256 * 256 + 256) + 256 * 8 + 8


def test_ctypes_structures_match_the_header_layout(tmp_path):
    # the binding's ctypes mirrors of the header's structs: same size and the
    # same offset for every field, as a C compiler lays them out from
    # include/hmle.h (gcc on this host; the layout rules are the platform ABI's)
    import ctypes as C
    import subprocess
    from paper_2104_07146_gb300 import hmle
    pairs = {"hmle_opts": hmle.Opts, "hmle_fit_opts": hmle.FitOpts, "hmle_theta": hmle.Theta,
             "hmle_tree_info": hmle.TreeInfo, "hmle_task": hmle.Task, "hmle_retry_info": hmle.RetryInfo,
             "hmle_tune_result": hmle.TuneResult, "hmle_eval_info": hmle.EvalInfo}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "hmle.h"', "int main(void) {"]
    for cname, cls in pairs.items():
        lines.append('printf("%s size %%zu\\n", sizeof(%s));' % (cname, cname))
        for f in cls._fields_:
            lines.append('printf("%s %s %%zu\\n", offsetof(%s, %s));' % (cname, f[0], cname, f[0]))
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.splitlines():
        a, b, v = line.split()
        got[(a, b)] = int(v)
    for cname, cls in pairs.items():
        assert got[(cname, "size")] == C.sizeof(cls), cname
        for f in cls._fields_:
            assert got[(cname, f[0])] == getattr(cls, f[0]).offset, (cname, f[0])


def _prototypes():
    """name -> list of parameter declarations of every function the header
    declares."""
    src = open(os.path.join(ROOT, "include", "hmle.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    out = {}
    for m in re.finditer(r"\b(hmle_[a-z_]+)\s*\(([^;{]*?)\)\s*;", src):
        params = [p.strip() for p in m.group(2).split(",") if p.strip() and p.strip() != "void"]
        out[m.group(1)] = params
    return out


def test_binding_signatures_match_the_header():
    # every ctypes signature the binding sets has the header's arity, and each
    # argument's kind (pointer, 64- or 32-bit integer, double, float) matches
    from paper_2104_07146_gb300 import hmle
    L = hmle.lib()
    protos = _prototypes()
    checked = 0
    for name, params in protos.items():
        fn = getattr(L, name)
        if fn.argtypes is None:
            continue
        assert len(fn.argtypes) == len(params), (name, params, fn.argtypes)
        for decl, at in zip(params, fn.argtypes):
            if "*" in decl or "[" in decl or "hmle_objective" in decl:
                assert at not in (C.c_int32, C.c_int64, C.c_double, C.c_float, C.c_uint64), (name, decl)
            elif re.search(r"\bu?int64_t\b", decl):
                assert at in (C.c_int64, C.c_uint64), (name, decl)
            elif re.search(r"\bu?int32_t\b", decl):
                assert at in (C.c_int32, C.c_uint32), (name, decl)
            elif re.search(r"\bdouble\b", decl):
                assert at is C.c_double, (name, decl)
            elif re.search(r"\bfloat\b", decl):
                assert at is C.c_float, (name, decl)
            else:
                raise AssertionError("unclassified parameter %r of %s" % (decl, name))
        checked += 1
    assert checked >= 40
