"""GPU parity of the division of eq. (10) where Q is small or vanishes (the guard; the paper
assumes Q > 0), through the C ABI, against the FP64 oracle's rule: output = input pixel when
|Q| < 1e-12 Qabs or Qabs = 0 (Qabs = the sum of the absolute terms of Q), else P/Q + t_c.

The exact forms take that decision in FP64: pixels their own arithmetic cannot resolve are
recomputed from the input in FP64 (n_refined).  So, with r = |Q|/Qabs from the oracle:
  * pixels with Qabs = 0 or r < 1e-14 are guarded on the GPU: output = input, bit for bit;
  * pixels with r > 1e-9 are not: n_guarded lies between the two oracle counts;
  * refined pixels (surely those with r far below the form's flag threshold) match the
    oracle's output to 1e-3 although they are ill-conditioned: in FP64 below 1e-2 (and
    always for the FP32 forms), in FP32 from the input above it (the 16-bit forms);
  * n_illcond (FP64 for refined pixels) lies between the oracle's counts at 0.9e-3 and 1.1e-3.
The recursive form decides on its FP32 sums (guarded below 2^-17 Qabs, their resolution), so
it is held to the bands r < 1e-8 (guarded) and r > 1e-4 (not guarded) against its twin.
A non-convergent fit (sigma_r = 8, N = 10, mu = 254) makes Q cancel at many pixels; a block
of value 1000 (far outside [0, 255]) makes every channel underflow, Qabs = 0.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, synth

pytestmark = pytest.mark.gpu

EXACT = [("plain", "fp32", 1e-3), ("fused", "fp32", 1e-3), ("fused_tc", "bf16", 1 / 16),
         ("fused_tc", "fp16", 1 / 128)]


def guard_image(H, W, seed, block=True):
    f = synth.rects_image(H, W, n_rects=10, noise_std=10.0, seed=seed).astype(np.float32)
    if block:
        f[10:40, W - 50:W - 14] = 1000.0
    return f


def run(f, ss, sr, N, form, prec):
    plan = api.GCPlan(f.shape[0], f.shape[1], ss, sr, N, form=form, precision=prec)
    ws = plan.workspace("fwd")
    out = plan.forward(torch.from_numpy(f).cuda(), ws=ws)
    torch.cuda.synchronize()
    return out.cpu().numpy(), plan.diagnostics(ws)


def ratio(aux):
    Qa = aux["Qabs"]
    with np.errstate(invalid="ignore", divide="ignore"):
        r = np.where(Qa > 0, np.abs(aux["Q"]) / Qa, 0.0)
    return r


@pytest.mark.parametrize("form,prec,flag", EXACT)
@pytest.mark.parametrize("H,W,ss", [(150, 200, 1.0), (133, 171, 4.0)])
def test_exact_forms_guard_like_the_oracle(form, prec, flag, H, W, ss):
    sr, N = 8.0, 10
    f = guard_image(H, W, seed=H + W)
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    r = ratio(aux)
    deep = (aux["Qabs"] == 0.0) | (r < 1e-14)
    loose = (aux["Qabs"] == 0.0) | (r < 1e-9)
    assert deep.sum() >= 50                        # the block's interior at least
    out, d = run(f, ss, sr, N, form, prec)
    assert d["error_flags"] == 0
    assert np.array_equal(out[deep], f[deep]), "deeply guarded pixels must return the input"
    assert deep.sum() <= d["n_guarded"] <= loose.sum(), (deep.sum(), d["n_guarded"], loose.sum())
    # refined: every pixel the form's own arithmetic cannot resolve (surely those far below its
    # flag threshold), recomputed in FP64: the oracle's output although ill-conditioned
    sure = (r < flag / 8) & ~loose
    assert sure.sum() >= 20
    # (more are refined where the form's channels underflow, e.g. FP32 at |u| > 0.84 when sigma_r = 8)
    assert d["n_refined"] >= (r < flag / 8).sum()
    # the FP64 tier takes every listed pixel of the FP32 forms, and of the 16-bit forms those an
    # FP32 recomputation leaves below 1e-2 Qabs
    assert d["n_refined_fp64"] >= ((r < min(5e-3, flag / 8)) | (aux["Qabs"] == 0.0)).sum()
    if prec == "fp32":
        assert d["n_refined_fp64"] == d["n_refined"]
    err = np.abs(out.astype(np.float64) - ref)
    Q = np.maximum(np.abs(aux["Q"]), 1e-300)
    # both sides in FP64: within the first-order rounding bound of P/Q at FP64 (with margin)
    bound64 = 1e-13 * (aux["Pabs"] + np.abs(aux["P"]) / Q * aux["Qabs"]) / Q + 1e-3
    assert np.all(err[sure] <= bound64[sure]), float(np.max(err[sure] - bound64[sure]))
    lo = ((r < 0.9e-3) & ~loose).sum()
    hi = ((r < 1.1e-3) & ~loose).sum()
    assert lo <= d["n_illcond"] <= hi, (lo, d["n_illcond"], hi)
    if prec == "bf16":
        # listed and settled by the FP32 recomputation: within its first-order rounding bound
        mid = (r >= 2e-2) & (r < flag / 2)
        assert mid.sum() >= 20
        bound32 = 1e-5 * (aux["Pabs"] + np.abs(aux["P"]) / Q * aux["Qabs"]) / Q + 1e-3
        assert np.all(err[mid] <= bound32[mid]), float(np.max(err[mid] - bound32[mid]))
    if prec == "fp32":
        # the rest is divided in FP32: within the first-order rounding bound of P/Q
        bound = 4e-6 * (aux["Pabs"] + np.abs(aux["P"]) / Q * aux["Qabs"]) / Q + 1e-3
        rest = ~loose & ~sure
        assert np.all(err[rest] <= bound[rest]), float(np.max(err[rest] - bound[rest]))


@pytest.mark.parametrize("form,prec,flag", EXACT)
def test_no_refinement_where_the_fit_converges(form, prec, flag):
    """sigma_r = 50, N = 20 (the benchmark's parameters): no pixel comes near the thresholds."""
    f = synth.edge_smooth_image(180, 260, noise_std=5.0, seed=3)
    ref = oracle.gcf(f, 3.0, 50.0, 20)
    out, d = run(f, 3.0, 50.0, 20, form, prec)
    assert d["n_refined"] == 0 and d["n_guarded"] == 0 and d["n_illcond"] == 0
    tol = {"fp32": 1e-3, "bf16": 0.5, "fp16": 0.05}[prec]
    assert np.abs(out.astype(np.float64) - ref).max() <= tol


def test_recursive_form_guards_on_its_fp32_sums():
    sr, N, ss = 8.0, 10, 2.0
    # every pixel far outside [0, 255]: every channel is 0 on both sides, every pixel guarded
    f = np.full((40, 50), 1000.0, dtype=np.float32)
    out, d = run(f, ss, sr, N, "recursive", "fp32")
    assert d["n_guarded"] == f.size and np.array_equal(out, f)
    # the non-convergent fit: few pixels near the band, none guarded beyond it (the infinite
    # impulse response leaks into every window, so the twin's Qabs never vanishes here)
    f = guard_image(150, 200, seed=5, block=False)
    ref, aux = oracle.gcf(f, ss, sr, N, spatial="recursive", return_pq=True)
    r = ratio(aux)
    sure = (aux["Qabs"] == 0.0) | (r < 1e-8)
    maybe = (aux["Qabs"] == 0.0) | (r < 1e-4)
    out, d = run(f, ss, sr, N, "recursive", "fp32")
    assert d["n_refined"] == 0 and d["error_flags"] == 0
    assert np.array_equal(out[sure], f[sure])
    assert sure.sum() <= d["n_guarded"] <= maybe.sum(), (sure.sum(), d["n_guarded"], maybe.sum())


@pytest.mark.parametrize("form,prec", [("plain", "fp32"), ("fused_tc", "fp16")])
def test_refinement_off_decides_on_the_forms_own_sums(form, prec):
    """BF_OPT_REFINE = 0: no list and no second launch; the guard is taken on the form's own
    sums at 2^-17 Qabs, like the recursive form."""
    sr, N, ss = 8.0, 10, 2.0
    f = guard_image(150, 200, seed=7)
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    r = ratio(aux)
    plan = api.GCPlan(150, 200, ss, sr, N, form=form, precision=prec, refine=False)
    on = api.GCPlan(150, 200, ss, sr, N, form=form, precision=prec)
    assert plan.workspace_bytes()[0] < on.workspace_bytes()[0]          # no list
    ws = plan.workspace("fwd")
    out = plan.forward(torch.from_numpy(f).cuda(), ws=ws).cpu().numpy()
    d = plan.diagnostics(ws)
    assert d["n_refined"] == 0 and d["error_flags"] == 0
    deep = aux["Qabs"] == 0.0                                           # every channel underflows
    assert np.array_equal(out[deep], f[deep])
    assert d["n_guarded"] >= deep.sum()


def test_static_forward_refines_like_the_workspace_forward():
    """The allocation-free entry point runs the same forward, refinement included."""
    from paper_1605_02178_gb300 import bfgc
    f = guard_image(150, 200, seed=9)
    plan = api.GCPlan(150, 200, 1.0, 8.0, 10, form="fused_tc", precision="bf16")
    ft = torch.from_numpy(f).cuda()
    a = plan.forward(ft)
    b = bfgc.bf_gc_forward_static(plan.handle, ft, torch.empty_like(ft))
    torch.cuda.synchronize()
    assert torch.equal(a, b)
