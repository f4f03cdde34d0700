"""CPU checks of the fused FP32 form's host logic (BF_FORM_FUSED): option values, workspace
size (one set of C FP32 channel planes, half of the plain form's two, then the FP64
refinement list of one 32-bit index per pixel), and the argument checks that return before
any CUDA call.  No kernel is launched here."""
import ctypes

import pytest

from paper_1605_02178_gb300 import bfgc as B
from paper_1605_02178_gb300.api import GCPlan


def _plane(H, W):
    return -(-H * W // 64) * 64


@pytest.mark.parametrize("H,W,N", [(1, 1, 4), (333, 517, 10), (2160, 3840, 20)])
def test_fused_workspace_is_one_set_of_planes(H, W, N):
    C = N + 2
    fused = GCPlan(H, W, 5.0, 30.0, N, form="fused").workspace_bytes()[0]
    plain = GCPlan(H, W, 5.0, 30.0, N, form="plain").workspace_bytes()[0]
    lst = -(-H * W * 4 // 256) * 256
    assert fused == 256 + C * _plane(H, W) * 4 + lst
    assert plain == 256 + 2 * C * _plane(H, W) * 4 + lst


def test_form_option_values():
    p = B.bf_gc_plan(50, 60, 3.0, 30.0, 8)
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_FUSED)
        assert B.bf_gc_plan_info(p).form == B.BF_FORM_FUSED
        for bad in (-1, 5, 4.5):
            with pytest.raises(B.BfError) as e:
                B.bf_gc_plan_set(p, B.BF_OPT_FORM, bad)
            assert e.value.status == B.BF_ERR_INVALID_ARG
    finally:
        B.bf_gc_plan_destroy(p)


@pytest.mark.parametrize("sigma_s,precision", [(3.0, B.BF_PREC_BF16), (3.0, B.BF_PREC_FP16), (58.0, B.BF_PREC_FP32)])
def test_unsupported_before_any_cuda_call(sigma_s, precision):
    """16-bit storage, or R = 174 (past the form's shared-memory windows): BF_ERR_UNSUPPORTED
    from bf_gc_forward, with fake device pointers that are never touched."""
    p = B.bf_gc_plan(64, 64, sigma_s, 50.0, 6)
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_FUSED)
        B.bf_gc_plan_set(p, B.BF_OPT_PRECISION, precision)
        st = B.lib().bf_gc_forward(p, ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20),
                                   ctypes.c_void_p(4 << 20), ctypes.c_size_t(1 << 30), None)
        assert st == B.BF_ERR_UNSUPPORTED
    finally:
        B.bf_gc_plan_destroy(p)


def test_largest_supported_radius_passes_the_checks():
    """R = 173 is accepted: the call gets past the form check to the workspace check."""
    p = B.bf_gc_plan(64, 64, 57.6, 50.0, 6)
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_FUSED)
        assert B.bf_gc_plan_info(p).R == 173
        st = B.lib().bf_gc_forward(p, ctypes.c_void_p(1 << 20), ctypes.c_void_p(2 << 20),
                                   ctypes.c_void_p(4 << 20), ctypes.c_size_t(16), None)
        assert st == B.BF_ERR_WORKSPACE
    finally:
        B.bf_gc_plan_destroy(p)
