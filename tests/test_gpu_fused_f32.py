"""GPU checks of the fused FP32 form (BF_FORM_FUSED: build + row pass, column pass + ratio on
the FP32 ALUs), called through the C ABI.

Every output of this form takes the same FP32 operations in the same order as in the plain
form, so the two are compared bit for bit (outputs and the guard / ill-conditioning counters)
over ragged sizes, windows wider than the image, the largest supported radius, small sigma_r
(guarded pixels), the Taylor coefficients and a custom intensity range.  Against the FP64
oracle the form is held to the FP32 tolerance, 1e-3 max-abs, at conditioned pixels.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, batch as BT, bfgc as B, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _run(f, ss, sr, N, form, **opts):
    plan = api.GCPlan(f.shape[0], f.shape[1], ss, sr, N, form=form, precision="fp32", **opts)
    ws = plan.workspace("fwd", f.device)
    out = plan.forward(f, torch.empty_like(f), ws)
    diag = plan.diagnostics(ws)
    torch.cuda.synchronize()
    return out, diag, plan


CASES = [
    # H, W, sigma_s, sigma_r, N, options
    (1, 1, 1.0, 50.0, 16, {}),
    (1, 37, 2.0, 50.0, 12, {}),
    (5, 3, 3.0, 50.0, 12, {}),
    (40, 33, 10.0, 50.0, 16, {}),          # window wider than the image: repeated reflection
    (97, 131, 2.0, 50.0, 12, {}),
    (300, 517, 10.0, 50.0, 20, {}),        # several tiles each way, ragged, W % 4 != 0
    (257, 1029, 4.0, 30.0, 28, {}),        # sigma_r = 30, N = 28
    (64, 384, 5.0, 60.0, 10, {}),          # whole tiles, W % 4 == 0
    (200, 96, 29.0, 50.0, 8, {}),          # R = 87
    (130, 250, 57.6, 50.0, 6, {}),         # R = 173, the largest radius of the form
    (120, 160, 3.0, 8.0, 10, {}),          # small sigma_r: guarded and ill-conditioned pixels
    (90, 77, 4.0, 40.0, 9, {"poly": "taylor"}),
    (66, 130, 3.0, 20.0, 12, {"L": 10.0, "U": 200.0}),
    (33, 70, 2.0, 120.0, 62, {}),          # N = 62: 64 channels, the most a plan takes
]


@pytest.mark.parametrize("H,W,ss,sr,N,opts", CASES)
def test_fused_equals_plain_bit_for_bit(H, W, ss, sr, N, opts):
    f = torch.from_numpy(synth.edge_smooth_image(H, W, noise_std=5.0, seed=H * 7 + W)).to(DEV)
    out_p, diag_p, _ = _run(f, ss, sr, N, "plain", **opts)
    out_f, diag_f, plan = _run(f, ss, sr, N, "fused", **opts)
    assert plan.info["form"] == B.BF_FORM_FUSED
    assert torch.equal(out_f, out_p)
    assert diag_f["n_guarded"] == diag_p["n_guarded"] and diag_f["n_illcond"] == diag_p["n_illcond"]
    assert diag_f["error_flags"] == 0


@pytest.mark.parametrize("H,W,ss,sr,N", [(97, 131, 2.0, 50.0, 12), (300, 257, 3.0, 50.0, 20),
                                          (130, 70, 3.0, 30.0, 28), (40, 33, 10.0, 50.0, 16),
                                          (256, 256, 10.0, 50.0, 20)])
def test_fused_matches_oracle(H, W, ss, sr, N):
    f = synth.rects_image(H, W, n_rects=8, noise_std=10.0, seed=H * 1000 + W)
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    out, _, plan = _run(torch.from_numpy(f).to(DEV), ss, sr, N, "fused")
    assert plan.info["fit_err"] <= 1e-2
    cond = aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300)
    mask = cond <= 1e4
    assert mask.mean() > 0.99
    err = np.abs(out.cpu().numpy().astype(np.float64) - ref)
    assert err[mask].max() <= 1e-3


def test_fused_at_uhd_sampled_against_oracle():
    """The 4K workload (3840x2160, sigma_s = 10, sigma_r = 50, N = 20) in the launch
    configuration the benchmark times, at sampled pixels."""
    wl = synth.workload("uhd")
    f = wl["f"]
    H, W = f.shape
    out, diag, _ = _run(torch.from_numpy(f).to(DEV), 10.0, 50.0, 20, "fused")
    rng = np.random.default_rng(11)
    idx = np.concatenate([[0, W - 1, (H - 1) * W, H * W - 1], rng.integers(0, H * W, 60)])
    ref = oracle.gcf_at(f, idx, 10.0, 50.0, 20)
    assert np.abs(out.cpu().numpy().reshape(-1)[idx].astype(np.float64) - ref).max() <= 1e-3
    assert diag["error_flags"] == 0


def test_fused_limits():
    f = torch.zeros(64, 64, device=DEV)
    with pytest.raises(B.BfError) as e:
        api.GCPlan(64, 64, 58.0, 50.0, 6, form="fused").forward(f)       # R = 174
    assert e.value.status == B.BF_ERR_UNSUPPORTED
    with pytest.raises(B.BfError) as e:
        api.GCPlan(64, 64, 3.0, 50.0, 6, form="fused", precision="bf16").forward(f)
    assert e.value.status == B.BF_ERR_UNSUPPORTED


def test_fused_backward_equals_plain():
    """The adjoint recomputes the channels with the plain kernels for every form, so the
    gradients of a fused-form plan equal those of a plain-form plan."""
    H, W = 70, 90
    f = torch.from_numpy(synth.edge_smooth_image(H, W, seed=3)).to(DEV)
    w = torch.from_numpy(np.random.default_rng(4).standard_normal((H, W)).astype(np.float32)).to(DEV)
    gp = api.GCPlan(H, W, 3.0, 40.0, 10, form="plain").backward(f, w)
    gq = api.GCPlan(H, W, 3.0, 40.0, 10, form="fused").backward(f, w)
    torch.cuda.synchronize()
    assert torch.equal(gp[0], gq[0]) and torch.equal(gp[1], gq[1])


def test_fused_batch_equals_per_image():
    specs = [
        {"H": 64, "W": 64, "sigma_s": 2.0, "sigma_r": 50.0, "N": 4, "seed": 1},
        {"H": 1, "W": 37, "sigma_s": 3.0, "sigma_r": 40.0, "N": 8, "seed": 2},
        {"H": 300, "W": 517, "sigma_s": 10.0, "sigma_r": 50.0, "N": 12, "seed": 4},
        {"H": 77, "W": 600, "sigma_s": 4.5, "sigma_r": 55.0, "N": 6, "seed": 6},
        {"H": 5, "W": 3, "sigma_s": 3.0, "sigma_r": 50.0, "N": 12, "seed": 9},
    ]
    fs = [torch.from_numpy(synth.edge_smooth_image(s["H"], s["W"], noise_std=5.0, seed=s["seed"])).to(DEV)
          for s in specs]
    outs = BT.GCBatch(specs, form="fused", precision="fp32", branches=3).forward(fs)
    torch.cuda.synchronize()
    for s, f, o in zip(specs, fs, outs):
        ref = api.GCPlan(s["H"], s["W"], s["sigma_s"], s["sigma_r"], s["N"], form="plain").forward(f)
        torch.cuda.synchronize()
        assert torch.equal(o, ref)
