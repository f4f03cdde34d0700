"""Checks on the GPU that need no fault: reads of unwritten workspace memory and races.

* Every form runs once on a zeroed workspace and once on a workspace whose every byte is
  0xFF (a NaN in FP32, BF16 and FP16 alike); the outputs and diagnostics must agree bit for
  bit, so no kernel reads workspace memory that the same forward did not write first.
* The tensor-core row pass has four kernels (BF_OPT_TILE_W 0, 64, 128, 256) that split the
  work differently over CTAs and warps; three of them sum the same products in the same
  order and must agree bit for bit on repeated runs.
"""
import numpy as np
import pytest
import torch

from paper_1605_02178_gb300 import api, synth

pytestmark = pytest.mark.gpu

FORMS = [("plain", "fp32"), ("fused", "fp32"), ("fused_tc", "bf16"), ("fused_tc", "fp16"), ("recursive", "fp32")]


@pytest.mark.parametrize("form,prec", FORMS)
@pytest.mark.parametrize("H,W,ss,sr,N", [(300, 257, 3.0, 50.0, 12), (97, 131, 10.0, 8.0, 10)])
def test_forward_ignores_what_the_workspace_held(form, prec, H, W, ss, sr, N):
    f = torch.from_numpy(synth.rects_image(H, W, n_rects=8, noise_std=10.0, seed=H + W)).cuda()
    plan = api.GCPlan(H, W, ss, sr, N, form=form, precision=prec)
    fwd = plan.workspace_bytes()[0]
    outs, diags = [], []
    for fill in (0x00, 0xFF, 0x00, 0xFF):
        ws = torch.full((fwd,), fill, dtype=torch.uint8, device="cuda")
        outs.append(plan.forward(f, ws=ws))
        diags.append(plan.diagnostics(ws))
    torch.cuda.synchronize()
    for o, d in zip(outs[1:], diags[1:]):
        assert torch.equal(o, outs[0])
        assert d == diags[0]
    assert torch.isfinite(outs[0]).all()


def test_row_pass_kernels_agree_on_repeated_runs():
    H, W = 260, 700
    f = torch.from_numpy(synth.edge_smooth_image(H, W, noise_std=5.0, seed=8)).cuda()
    ref = None
    for tw in (64, 128, 256):
        plan = api.GCPlan(H, W, 3.0, 50.0, 16, form="fused_tc", precision="bf16", tile_w=tw)
        for _ in range(2):
            o = plan.forward(f)
            torch.cuda.synchronize()
            if ref is None:
                ref = o.clone()
            assert torch.equal(o, ref), f"tile width {tw}"
    plan = api.GCPlan(H, W, 3.0, 50.0, 16, form="fused_tc", precision="bf16")
    a, b = plan.forward(f), plan.forward(f)
    torch.cuda.synchronize()
    assert torch.equal(a, b)
    assert float((a - ref).abs().max()) <= 0.05          # the default kernel sums in another order
    assert np.isfinite(a.cpu().numpy()).all()


def test_range_check_counts_planted_pixels():
    """bf_check_range against numpy's count: pixels outside [L, U] and non-finite ones planted at
    seeded positions, on an odd-sized image (scalar tail) and through an offset view (no 16-byte
    alignment)."""
    from paper_1605_02178_gb300 import bfgc
    rng = np.random.default_rng(3)
    H, W = 257, 131
    f = rng.uniform(0.0, 255.0, (H, W)).astype(np.float32)
    idx = rng.choice(H * W, 400, replace=False)
    f.reshape(-1)[idx[:150]] = rng.uniform(256.0, 400.0, 150).astype(np.float32)
    f.reshape(-1)[idx[150:300]] = rng.uniform(-100.0, -0.5, 150).astype(np.float32)
    f.reshape(-1)[idx[300:350]] = np.nan
    f.reshape(-1)[idx[350:400]] = np.inf * np.sign(rng.uniform(-1, 1, 50))
    fin = np.isfinite(f)
    want = (int(np.sum(fin & ((f < 0.0) | (f > 255.0)))), int(np.sum(~fin)))
    t = torch.from_numpy(f).cuda()
    assert bfgc.bf_check_range(t, 0.0, 255.0) == want == (300, 100)
    # the same pixels one float off a 16-byte boundary
    buf = torch.empty(H * W + 1, dtype=torch.float32, device="cuda")
    buf[1:] = t.reshape(-1)
    assert bfgc.bf_check_range(buf[1:].view(H, W), 0.0, 255.0) == want
    # a clean image
    assert bfgc.bf_check_range(torch.full((5, 3), 7.0, device="cuda"), 0.0, 255.0) == (0, 0)
