"""GPU checks of the persistent batched forward (bf_gc_batch_create_persistent): one launch of
the batched row pass and one of the batched column pass over a device work list of
(image, tile) items.

Each image is filtered at the batch's window block count a with its own taps, so it must
agree with its own tensor-core forward up to the FP32 summation order of the banded products
(one 16-bit rounding of a channel at most), and with the FP64 oracle within the channel
storage's bound (BF16 0.5, FP16 0.05 max-abs) at sampled pixels of the images whose
range-kernel fit converges.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, batch as BT, synth
from paper_1605_02178_gb300.bfgc import BfError

pytestmark = pytest.mark.gpu

DEV = "cuda"
BOUND = {"bf16": 0.5, "fp16": 0.05}

# mixed sizes (ragged, tiny, rows not a multiple of 4 floats, wider than a tile) and radii over
# a = 1..3 in one batch, so that every image is laid out at a = 3 with zero taps beyond its R
SPECS = [
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


def _images(specs):
    return [torch.from_numpy(synth.edge_smooth_image(s["H"], s["W"], noise_std=5.0, seed=s["seed"])).to(DEV)
            for s in specs]


def _convergent(s):
    return api.GCPlan(s["H"], s["W"], s["sigma_s"], s["sigma_r"], s["N"]).info["fit_err"] <= 1e-2


def _check(specs, fs, outs, precision, per_image_tol, samples=12, seed=5):
    rng = np.random.default_rng(seed)
    checked = 0
    for s, f, o in zip(specs, fs, outs):
        assert torch.isfinite(o).all()
        # where the fit diverges the output is no filter, and the per-image forward divides its
        # ill-conditioned pixels in FP64: nothing to compare
        if not _convergent(s):
            continue
        plan = api.GCPlan(s["H"], s["W"], s["sigma_s"], s["sigma_r"], s["N"], form="fused_tc", precision=precision)
        ref_tc = plan.forward(f)
        torch.cuda.synchronize()
        assert float((o - ref_tc).abs().max()) <= per_image_tol, s
        checked += 1
        idx = rng.integers(0, s["H"] * s["W"], samples)
        ref = oracle.gcf_at(f.cpu().numpy(), idx, s["sigma_s"], s["sigma_r"], s["N"])
        assert np.abs(o.cpu().numpy().reshape(-1)[idx] - ref).max(initial=0.0) <= BOUND[precision], s
    return checked


@pytest.mark.parametrize("precision", ["bf16", "fp16"])
def test_persistent_batch_matches_per_image_and_oracle(precision):
    fs = _images(SPECS)
    bt = BT.GCBatch(SPECS, form="fused_tc", precision=precision, mode="persistent")
    outs = bt.forward(fs)
    torch.cuda.synchronize()
    d = bt.diagnostics()
    assert d["error_flags"] == 0
    assert _check(SPECS, fs, outs, precision, BOUND[precision] / 2) >= 4
    # the captured graph again, on the same tensors: the same bits; then new output tensors
    again = [torch.full_like(o, float("nan")) for o in outs]
    bt.forward(fs, again)
    torch.cuda.synchronize()
    assert all(torch.equal(a, o) for a, o in zip(again, outs))
    assert bt.info()[1] == 2


def test_persistent_aligned_batch():
    """Every row a multiple of 16 bytes (W % 4 == 0): the batch takes the instantiations with
    16-byte accesses only (the mixed batches above take those that also handle other pitches)."""
    specs = [dict(s, W=max(4, s["W"] - s["W"] % 4)) for s in SPECS]
    assert all(s["W"] % 4 == 0 for s in specs)
    fs = _images(specs)
    bt = BT.GCBatch(specs, form="fused_tc", precision="bf16", mode="persistent")
    outs = bt.forward(fs)
    torch.cuda.synchronize()
    assert bt.diagnostics()["error_flags"] == 0
    assert _check(specs, fs, outs, "bf16", BOUND["bf16"] / 2) >= 4


def test_persistent_batch_rejects_misaligned_pointers():
    """Inputs and outputs must start on 16-byte boundaries (a view one float into a buffer does
    not): the call fails before any launch."""
    specs = SPECS[:3]
    fs = _images(specs)
    buf = torch.empty(specs[0]["H"] * specs[0]["W"] + 1, device=DEV)
    shifted = buf[1:].view(specs[0]["H"], specs[0]["W"])
    shifted.copy_(fs[0])
    bt = BT.GCBatch(specs, form="fused_tc", precision="bf16", mode="persistent")
    with pytest.raises(BfError):
        bt.forward([shifted] + fs[1:])


def test_persistent_uneven_batch_against_oracle():
    """48 images of the uneven batch workload (sizes 64..2048, own sigma_s, sigma_r and N)."""
    specs = synth.batch_specs(256, seed=4)[:48]
    fs = _images(specs)
    bt = BT.GCBatch(specs, form="fused_tc", precision="bf16", mode="persistent")
    outs = bt.forward(fs)
    torch.cuda.synchronize()
    assert bt.diagnostics()["error_flags"] == 0
    assert _check(specs, fs, outs, "bf16", 0.25, samples=8) >= 10


def test_persistent_batch_refuses_what_it_cannot_run():
    f = [{"H": 64, "W": 64, "sigma_s": 30.0, "sigma_r": 50.0, "N": 8, "seed": 1}]     # R = 90 > 64
    with pytest.raises(BfError):
        BT.GCBatch(f, form="fused_tc", precision="bf16", mode="persistent")
    with pytest.raises(BfError):
        BT.GCBatch(SPECS[:2], form="plain", precision="fp32", mode="persistent")


@pytest.mark.parametrize("stall,flag", [(1, 4), (2, 8)])
def test_persistent_batch_wait_runs_out_and_recovers(stall, flag):
    """The bounded waits of the batched passes: with BF_OPT_STALL on the first plan (1: the row
    pass's first tile is never handed to the MMA issuer; 2: the column pass's first stage is
    never loaded) and a 2 ms wait limit, the waits run out, the kernels return and the pass's
    error flag is set; a following batch without the stall is whole again."""
    from paper_1605_02178_gb300 import bfgc as B
    specs = SPECS[:4]
    fs = _images(specs)
    bt = BT.GCBatch(specs, form="fused_tc", precision="bf16", mode="persistent")
    B.bf_gc_plan_set(bt.plans[0].handle, B.BF_OPT_WAIT_US, 2000)
    B.bf_gc_plan_set(bt.plans[0].handle, B.BF_OPT_STALL, stall)
    bt.forward(fs)
    torch.cuda.synchronize()
    assert bt.diagnostics()["error_flags"] & flag
    ok = BT.GCBatch(specs, form="fused_tc", precision="bf16", mode="persistent")
    outs = ok.forward(fs)
    torch.cuda.synchronize()
    assert ok.diagnostics()["error_flags"] == 0
    assert _check(specs, fs, outs, "bf16", BOUND["bf16"] / 2) >= 1
