"""BF_FORM_AUTO: the form chosen from the window radius R = ceil(3 sigma_s) and the storage
precision (host logic, checked on the CPU through bf_gc_plan_info; no kernel is launched),
and, on the GPU, that an AUTO plan computes exactly what the chosen form computes."""
import numpy as np
import pytest
import torch

from paper_1605_02178_gb300 import api, bfgc as B, synth


def _form(sigma_s, precision, N=8):
    p = B.bf_gc_plan(64, 64, sigma_s, 40.0, N)
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_AUTO)
        B.bf_gc_plan_set(p, B.BF_OPT_PRECISION, B.PRECISIONS[precision])
        info = B.bf_gc_plan_info(p)
        return info.form, info.R
    finally:
        B.bf_gc_plan_destroy(p)


@pytest.mark.parametrize("sigma_s,precision,want", [
    (10.0, "fp32", B.BF_FORM_FUSED), (46.6, "fp32", B.BF_FORM_FUSED),          # R = 30, 140
    (46.7, "fp32", B.BF_FORM_RECURSIVE), (64.0, "fp32", B.BF_FORM_RECURSIVE),  # R = 141, 192
    (10.0, "bf16", B.BF_FORM_FUSED_TC), (42.0, "fp16", B.BF_FORM_FUSED_TC),     # R = 30, 126
    (42.7, "bf16", B.BF_FORM_RECURSIVE), (64.0, "fp16", B.BF_FORM_RECURSIVE),   # R = 129, 192
])
def test_auto_form_follows_radius_and_precision(sigma_s, precision, want):
    form, R = _form(sigma_s, precision)
    assert form == want, (sigma_s, precision, R, form)
    assert (R <= B.BF_AUTO_FP32_EXACT_MAX_R) == (form == B.BF_FORM_FUSED) or precision != "fp32"


def test_auto_form_follows_precision_changes_and_explicit_forms():
    p = B.bf_gc_plan(64, 64, 10.0, 40.0, 8)
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_AUTO)
        assert B.bf_gc_plan_info(p).form == B.BF_FORM_FUSED
        B.bf_gc_plan_set(p, B.BF_OPT_PRECISION, B.BF_PREC_BF16)
        assert B.bf_gc_plan_info(p).form == B.BF_FORM_FUSED_TC
        B.bf_gc_plan_set(p, B.BF_OPT_PRECISION, B.BF_PREC_FP32)
        assert B.bf_gc_plan_info(p).form == B.BF_FORM_FUSED
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_RECURSIVE)     # an explicit form ends AUTO
        B.bf_gc_plan_set(p, B.BF_OPT_PRECISION, B.BF_PREC_BF16)
        assert B.bf_gc_plan_info(p).form == B.BF_FORM_RECURSIVE
        with pytest.raises(B.BfError):                              # recursive is FP32-only outside AUTO
            B.bf_gc_workspace_size(p)
        with pytest.raises(B.BfError):
            B.bf_gc_plan_set(p, B.BF_OPT_FORM, 5)
    finally:
        B.bf_gc_plan_destroy(p)


def test_auto_recursive_with_16bit_storage_has_no_backward_but_a_forward_workspace():
    p = api.GCPlan(64, 64, 50.0, 40.0, 8, form="auto", precision="bf16")
    assert p.info["form"] == B.BF_FORM_RECURSIVE
    fwd, bwd = p.workspace_bytes()
    assert fwd > 0


@pytest.mark.gpu
@pytest.mark.parametrize("sigma_s,precision,form", [(10.0, "bf16", "fused_tc"), (50.0, "bf16", "recursive"),
                                                    (10.0, "fp32", "fused"), (50.0, "fp32", "recursive")])
def test_auto_plan_computes_the_chosen_form(sigma_s, precision, form):
    f = torch.from_numpy(synth.edge_smooth_image(150, 170, seed=21)).cuda()
    auto = api.GCPlan(150, 170, sigma_s, 50.0, 12, form="auto", precision=precision).forward(f)
    ref = api.GCPlan(150, 170, sigma_s, 50.0, 12, form=form,
                     precision=precision if form == "fused_tc" else "fp32").forward(f)
    torch.cuda.synchronize()
    assert torch.equal(auto, ref)
