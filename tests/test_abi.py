"""CPU-only checks of the C ABI: the library builds, loads and exports every entry point
declared in include/bfgc.h; host-side plan logic (argument checks, options, the FP64
coefficient fit) behaves as documented.  No kernel is launched here."""
import ctypes
import math
import os
import re
import subprocess

import numpy as np
import pytest

import oracle
from paper_1605_02178_gb300 import bfgc as B

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "bfgc.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bf_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_expected_entry_points():
    names = declared_functions()
    for must in ("bf_gc_plan", "bf_gc_forward", "bf_gc_backward", "bf_direct"):
        assert must in names
    assert set(names) == set(B.SIGNATURES), "binding and header disagree"


def test_library_exports_every_declared_symbol():
    lib = B.lib()
    for name in declared_functions():
        assert hasattr(lib, name), name
    out = subprocess.run(["nm", "-D", "--defined-only", B.LIB_PATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r"\bT\s+(\w+)$", out, flags=re.M))
    assert set(declared_functions()) <= exported
    assert not any(s.startswith("oracle_") for s in exported)     # no oracle code in the product


def test_library_does_not_link_the_oracle():
    out = subprocess.run(["ldd", B.LIB_PATH], capture_output=True, text=True).stdout
    assert "bfgc_oracle" not in out


@pytest.mark.parametrize("args", [
    (0, 10, 1.0, 10.0, 4), (10, 0, 1.0, 10.0, 4), (10, 10, 0.0, 10.0, 4), (10, 10, 1.0, -1.0, 4),
    (10, 10, 1.0, 10.0, 0), (10, 10, 1.0, 10.0, B.BF_MAX_N + 1), (10, 10, float("nan"), 10.0, 4)])
def test_plan_rejects_invalid_arguments(args):
    with pytest.raises(B.BfError) as e:
        B.bf_gc_plan(*args)
    assert e.value.status == B.BF_ERR_INVALID_ARG


def test_plan_rejects_window_beyond_limit():
    with pytest.raises(B.BfError) as e:
        B.bf_gc_plan(10, 10, 90.0, 10.0, 4)
    assert e.value.status == B.BF_ERR_UNSUPPORTED


def test_plan_options_and_info():
    p = B.bf_gc_plan(2160, 3840, 10.0, 50.0, 20)
    try:
        i = B.bf_gc_plan_info(p)
        assert (i.H, i.W, i.N, i.C, i.R) == (2160, 3840, 20, 22, 30)
        assert i.t_c == 127.5 and i.s_r == 127.5
        assert i.mu == pytest.approx(255.0 ** 2 / (4 * 50.0 ** 2), rel=1e-15)
        for opt, bad in [(B.BF_OPT_FORM, 7), (B.BF_OPT_PRECISION, 3), (B.BF_OPT_POLY, 2), (99, 0),
                         (B.BF_OPT_FORM, 0.5)]:
            with pytest.raises(B.BfError):
                B.bf_gc_plan_set(p, opt, bad)
        with pytest.raises(B.BfError):
            B.bf_gc_plan_set(p, B.BF_OPT_RANGE_U, -5.0)                 # U <= L
        fwd, bwd = B.bf_gc_workspace_size(p)
        assert fwd >= 2 * 22 * 2160 * 3840 * 4
        B.bf_gc_plan_set(p, B.BF_OPT_RANGE_L, 16.0)
        B.bf_gc_plan_set(p, B.BF_OPT_RANGE_U, 235.0)
        i = B.bf_gc_plan_info(p)
        assert i.t_c == pytest.approx(125.5) and i.s_r == pytest.approx(109.5)
    finally:
        B.bf_gc_plan_destroy(p)


@pytest.mark.parametrize("sr,N", [(50.0, 20), (30.0, 8), (60.0, 4), (25.0, 10), (40.0, 16)])
def test_plan_coefficients_match_oracle_fit(sr, N):
    """The library's FP64 fit (written separately) gives the oracle's c_n of eq. (19)
    up to the roundoff of the monomial conversion (relative to max |c~_n|)."""
    p = B.bf_gc_plan(64, 64, 3.0, sr, N)
    try:
        i = B.bf_gc_plan_info(p)
        ref = oracle.cheb_fit(N, i.mu)["c"] * i.mu ** np.arange(N + 1)
        got = np.array(i.c_tilde[: N + 1])
        assert np.max(np.abs(got - ref)) <= 1e-6 * np.abs(ref).max()
        assert i.kappa == pytest.approx(np.abs(ref).max(), rel=1e-6)
    finally:
        B.bf_gc_plan_destroy(p)


def test_taylor_option_gives_inverse_factorials():
    p = B.bf_gc_plan(8, 8, 1.0, 40.0, 9)
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_POLY, B.BF_POLY_TAYLOR)
        i = B.bf_gc_plan_info(p)
        assert np.allclose([i.c[n] for n in range(10)], [1 / math.factorial(n) for n in range(10)], rtol=1e-14)
    finally:
        B.bf_gc_plan_destroy(p)


def test_fit_error_reports_convergence():
    errs = []
    for N in (4, 8, 12, 16, 20):
        p = B.bf_gc_plan(8, 8, 1.0, 50.0, N)
        errs.append(B.bf_gc_plan_info(p).fit_err)
        B.bf_gc_plan_destroy(p)
    assert all(b < a for a, b in zip(errs, errs[1:])) and errs[-1] < 1e-8


def test_direct_rejects_bad_arguments_without_launching():
    assert B.lib().bf_direct(0, 4, 1.0, 1.0, ctypes.c_void_p(256), ctypes.c_void_p(256), None) == B.BF_ERR_INVALID_ARG
    assert B.lib().bf_direct(4, 4, 1.0, 1.0, ctypes.c_void_p(258), ctypes.c_void_p(256), None) == B.BF_ERR_INVALID_ARG


def header_constants():
    """Every BF_* constant the header defines (enum members and integer #defines)."""
    text = re.sub(r"/\*.*?\*/", "", open(HEADER).read(), flags=re.S)
    out = {}
    for body in re.findall(r"enum\s*\{(.*?)\}", text, flags=re.S):
        for name, value in re.findall(r"\b(BF_[A-Z0-9_]+)\s*=\s*(-?\d+)", body):
            out[name] = int(value)
    for name, value in re.findall(r"#define\s+(BF_[A-Z0-9_]+)\s+(-?\d+)\b", text):
        out[name] = int(value)
    return out


def test_binding_constants_equal_the_header():
    consts = header_constants()
    for must in ("BF_FORM_PLAIN", "BF_FORM_FUSED", "BF_FORM_FUSED_TC", "BF_FORM_RECURSIVE", "BF_FORM_AUTO",
                 "BF_OPT_FORM", "BF_OPT_TILE_W", "BF_PREC_FP16", "BF_AUTO_FP32_EXACT_MAX_R", "BF_MAX_N"):
        assert must in consts, must
    shared = [n for n in consts if hasattr(B, n)]
    assert len(shared) >= 20
    for name in shared:
        assert getattr(B, name) == consts[name], name
    assert set(B.FORMS.values()) == {v for n, v in consts.items() if n.startswith("BF_FORM_")}


def test_bench_roofline_model_names_the_profiled_kernels():
    """bench.py's per-kernel work model has an entry for every kernel the forward of each form
    marks for the profiler (plan.cpp), so no kernel's roofline is silently dropped."""
    import sys
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "paper_1605_02178_gb300", "csrc", "plan.cpp")).read()
    body = src[src.index("bf_status bf_gc_forward("):src.index("bf_status bf_gc_forward_host(")]
    forms = {"BF_FORM_PLAIN": "plain", "BF_FORM_FUSED": "fused", "BF_FORM_FUSED_TC": "fused_tc",
             "BF_FORM_RECURSIVE": "recursive"}
    switch = body[body.index("switch (p->form) {"):body.index("default:")]
    after = body[body.index("default:"):]
    common = set(re.findall(r'prof_mark\(p, "(\w+)"', after))      # launched after every refining form
    assert common == {"refine_fp64"}
    cases = re.split(r"\n\s*case (BF_FORM_[A-Z_]+): \{", switch)
    seen = set()
    for enum_name, block in zip(cases[1::2], cases[2::2]):
        marks = set(re.findall(r'prof_mark\(p, "(\w+)"', block))
        form = forms[enum_name]
        if form != "recursive":
            marks |= common
        prec = "fp32" if form != "fused_tc" else "bf16"
        assert marks and marks == set(bench.kernel_model(form, prec, 22, 30)), form
        seen.add(form)
    assert seen == set(forms.values())


def test_wait_stall_and_refine_options_are_checked():
    p = B.bf_gc_plan(64, 64, 2.0, 50.0, 8)
    try:
        for opt, bad in ((B.BF_OPT_WAIT_US, 0.5), (B.BF_OPT_WAIT_US, 2e7), (B.BF_OPT_STALL, 3),
                         (B.BF_OPT_STALL, 1.5), (B.BF_OPT_REFINE, 2), (B.BF_OPT_REFINE, -1)):
            with pytest.raises(B.BfError) as e:
                B.bf_gc_plan_set(p, opt, bad)
            assert e.value.status == B.BF_ERR_INVALID_ARG
        for opt, good in ((B.BF_OPT_WAIT_US, 2000.0), (B.BF_OPT_STALL, 2), (B.BF_OPT_STALL, 0),
                          (B.BF_OPT_REFINE, 0)):
            B.bf_gc_plan_set(p, opt, good)
        # without the refinement the forward workspace holds no list
        B.bf_gc_plan_set(p, B.BF_OPT_REFINE, 1)
        with_list = B.bf_gc_workspace_size(p)[0]
        B.bf_gc_plan_set(p, B.BF_OPT_REFINE, 0)
        assert B.bf_gc_workspace_size(p)[0] == with_list - 64 * 64 * 4
    finally:
        B.bf_gc_plan_destroy(p)


def test_plan_warns_when_the_range_fit_diverges():
    """A degree too low for exp on [-mu, mu] gives a kernel off by orders of magnitude: the
    plan says so; a convergent fit (sigma_r = 50, N = 20) stays silent."""
    import warnings
    from paper_1605_02178_gb300 import api
    with pytest.warns(RuntimeWarning, match="raise N"):
        p = api.GCPlan(64, 64, 3.0, 10.0, 5)
    assert p.info["fit_err"] >= api.FIT_DIVERGES
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        q = api.GCPlan(64, 64, 3.0, 50.0, 20)
    assert q.info["fit_err"] < 1e-6


def test_plan_warns_about_bf16_where_it_misses_the_bound():
    """sigma_r = 30, N = 28 (the paper's operating point, mu = 18): BF16 storage is flagged, FP16
    is not; sigma_r = 50 (mu = 6.5) is quiet for BF16."""
    import warnings
    from paper_1605_02178_gb300 import api
    with pytest.warns(RuntimeWarning, match="fp16"):
        api.GCPlan(64, 64, 3.0, 30.0, 28, form="fused_tc", precision="bf16")
    with warnings.catch_warnings():
        warnings.simplefilter("error")
        api.GCPlan(64, 64, 3.0, 30.0, 28, form="fused_tc", precision="fp16")
        api.GCPlan(64, 64, 3.0, 50.0, 20, form="fused_tc", precision="bf16")
