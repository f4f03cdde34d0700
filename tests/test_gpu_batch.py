"""GPU checks of batched filtering (bf_gc_batch_* through the C ABI) and of the row-pass
tile width.

A batch runs the same kernels as single-image forwards, so every image of a batch must
equal the per-image forward of its plan bit for bit, whatever the branch count, the branch
an image lands on and the row-pass tile width.  Against the per-image loop of the plain
FP32 kernels the tensor-core batch (BF16 storage) is held to the BF16 tolerance, 0.5
max-abs, at sampled pixels of the images whose range-kernel fit error is <= 1e-2, where
both are also checked against the FP64 oracle (1e-3 and 0.5).
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, autotune, batch as BT, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _images(specs):
    return [torch.from_numpy(synth.edge_smooth_image(s["H"], s["W"], noise_std=5.0, seed=s["seed"])).to(DEV)
            for s in specs]


def _per_image(specs, fs, form, precision):
    outs = []
    for s, f in zip(specs, fs):
        plan = api.GCPlan(s["H"], s["W"], s["sigma_s"], s["sigma_r"], s["N"], form=form, precision=precision,
                          tile_w=s.get("tile_w", 0))
        outs.append(plan.forward(f))
    torch.cuda.synchronize()
    return outs


# mixed sizes (ragged, tiny, wider than one tile), radii over a = 1..3 and channel counts
SMALL_SPECS = [
    {"H": 64, "W": 64, "sigma_s": 2.0, "sigma_r": 50.0, "N": 4, "seed": 1},
    {"H": 1, "W": 37, "sigma_s": 3.0, "sigma_r": 40.0, "N": 8, "seed": 2},
    {"H": 131, "W": 97, "sigma_s": 6.0, "sigma_r": 60.0, "N": 16, "seed": 3},
    {"H": 300, "W": 517, "sigma_s": 10.0, "sigma_r": 50.0, "N": 12, "seed": 4},
    {"H": 257, "W": 129, "sigma_s": 16.0, "sigma_r": 45.0, "N": 10, "seed": 5},
    {"H": 77, "W": 600, "sigma_s": 4.5, "sigma_r": 55.0, "N": 6, "seed": 6},
    {"H": 512, "W": 300, "sigma_s": 12.0, "sigma_r": 50.0, "N": 14, "seed": 7},
    {"H": 33, "W": 2048, "sigma_s": 2.5, "sigma_r": 60.0, "N": 5, "seed": 8},
    {"H": 5, "W": 3, "sigma_s": 3.0, "sigma_r": 50.0, "N": 12, "seed": 9},
]


@pytest.mark.parametrize("tw", [128, 256])
@pytest.mark.parametrize("H,W,ss,N,prec", [(300, 517, 10.0, 12, "bf16"), (131, 97, 6.0, 16, "fp16"),
                                           (64, 700, 16.0, 4, "bf16"), (257, 65, 4.0, 20, "bf16")])
def test_tile_width_does_not_change_the_result(H, W, ss, N, prec, tw):
    """The shared-memory-Toeplitz row pass gives the same bits at every tile width; the default
    (tensor-memory Toeplitz) row pass sums the same products in another order."""
    f = torch.from_numpy(synth.edge_smooth_image(H, W, seed=H + W)).to(DEV)
    ref = api.GCPlan(H, W, ss, 50.0, N, form="fused_tc", precision=prec, tile_w=64).forward(f)
    out = api.GCPlan(H, W, ss, 50.0, N, form="fused_tc", precision=prec, tile_w=tw).forward(f)
    dflt = api.GCPlan(H, W, ss, 50.0, N, form="fused_tc", precision=prec).forward(f)
    torch.cuda.synchronize()
    assert torch.equal(out, ref)
    assert (dflt - ref).abs().max().item() <= (0.5 if prec == "bf16" else 0.05)


@pytest.mark.parametrize("branches", [1, 3, 8])
@pytest.mark.parametrize("form,precision", [("fused_tc", "bf16"), ("fused_tc", "fp16"), ("plain", "fp32"),
                                            ("fused", "fp32")])
def test_batch_equals_per_image_forwards(form, precision, branches):
    fs = _images(SMALL_SPECS)
    ref = _per_image(SMALL_SPECS, fs, form, precision)
    bt = BT.GCBatch(SMALL_SPECS, form=form, precision=precision, branches=branches)
    outs = bt.forward(fs)
    torch.cuda.synchronize()
    for i, (o, r) in enumerate(zip(outs, ref)):
        assert torch.equal(o, r), f"image {i}"
    # replay of the captured graph on the same tensors, then a re-capture on new outputs
    for o in outs:
        o.fill_(-1.0)
    bt.forward(fs, outs)
    outs2 = bt.forward(fs)
    torch.cuda.synchronize()
    assert bt.info()[1] == 2
    for o, o2, r in zip(outs, outs2, ref):
        assert torch.equal(o, r) and torch.equal(o2, r)


def test_batch_with_mixed_tile_widths_equals_per_image():
    specs = [dict(s, tile_w=(0, 64, 128, 256)[i % 4]) for i, s in enumerate(SMALL_SPECS)]
    fs = _images(specs)
    ref = _per_image(specs, fs, "fused_tc", "bf16")
    outs = BT.GCBatch(specs, form="fused_tc", precision="bf16", branches=4).forward(fs)
    torch.cuda.synchronize()
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)


def test_autotuned_batch_equals_per_image(tmp_path):
    tuner = autotune.Autotuner(path=str(tmp_path / "tune.json"), reps=1)
    fs = _images(SMALL_SPECS)
    ref = _per_image(SMALL_SPECS, fs, "fused_tc", "bf16")
    bt = BT.GCBatch(SMALL_SPECS, form="fused_tc", precision="bf16", tuner=tuner)
    outs = bt.forward(fs)
    torch.cuda.synchronize()
    assert bt.branches in autotune.BRANCH_COUNTS
    for o, r in zip(outs, ref):
        assert torch.equal(o, r)
    cached = tuner.cached()
    assert cached["tile_w"] and len(cached["branches"]) == 1


def _convergent(spec):
    plan = api.GCPlan(spec["H"], spec["W"], spec["sigma_s"], spec["sigma_r"], spec["N"])
    return plan.info["fit_err"] <= 1e-2


def test_uneven_batch_against_plain_loop_and_oracle():
    """The uneven batch workload (sizes 64..2048, own sigma_s, sigma_r and N per image), 48 of
    its images: the tensor-core batch against the per-image loop of the plain kernels, and
    sampled pixels against the oracle."""
    specs = synth.batch_specs(256, seed=4)[:48]
    fs = _images(specs)
    plain = _per_image(specs, fs, "plain", "fp32")
    outs = BT.GCBatch(specs, form="fused_tc", precision="bf16", branches=8).forward(fs)
    torch.cuda.synchronize()
    rng = np.random.default_rng(5)
    checked = 0
    for s, f, o, p in zip(specs, fs, outs, plain):
        assert torch.isfinite(o).all()
        if not _convergent(s):
            continue
        checked += 1
        H, W = s["H"], s["W"]
        idx = rng.integers(0, H * W, 12)
        ref = oracle.gcf_at(f.cpu().numpy(), idx, s["sigma_s"], s["sigma_r"], s["N"])
        on = o.cpu().numpy().reshape(-1)
        pn = p.cpu().numpy().reshape(-1)
        assert np.abs(pn[idx] - ref).max(initial=0.0) <= 1e-3
        assert np.abs(on[idx] - ref).max(initial=0.0) <= 0.5
        assert np.abs(on[idx] - pn[idx]).max(initial=0.0) <= 0.5 + 1e-3
    assert checked >= 10
