"""GPU parity of the forward filter and of the exact filter against the FP64 oracle,
called through the C ABI on seeded synthetic images.

Tolerance (max-abs on the [0, 255] output): 1e-3 for the FP32 form, applied to pixels
whose denominator is conditioned (cond = sum|terms of Q| / |Q| <= 1e4) in
configurations whose range-kernel fit error is <= 1e-2.  Elsewhere (the
non-convergent degree/sigma_r pairs, where P and Q are sums with heavy cancellation)
the FP32 result is checked against the first-order rounding bound of P/Q,
    |err| <= eps (Pabs + |P/Q| Qabs) / |Q| + 1e-3,  eps = 4e-6 (about 32 FP32 ulps),
with Pabs, Qabs the sums of the absolute values of the terms of P and Q.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, bfgc, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _image(H, W, seed, noise=10.0):
    return synth.rects_image(H, W, n_rects=8, noise_std=noise, seed=seed)


def fp32_bound(aux, eps=4e-6):
    Q = np.maximum(np.abs(aux["Q"]), 1e-300)
    return eps * (aux["Pabs"] + np.abs(aux["P"]) / Q * aux["Qabs"]) / Q + 1e-3


def _gpu_forward(f, ss, sr, N, **opts):
    plan = api.GCPlan(f.shape[0], f.shape[1], ss, sr, N, **opts)
    out = plan.forward(torch.from_numpy(f).to(DEV))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), plan


CONDITIONED = [
    (97, 131, 2.0, 50.0, 12),
    (300, 257, 3.0, 50.0, 20),
    (64, 200, 5.0, 60.0, 10),
    (130, 70, 3.0, 30.0, 28),     # the paper's Table 2 operating point (sigma_r = 30, N = 28)
    (40, 33, 10.0, 50.0, 16),     # window wider than the image: repeated reflection
    (1, 37, 2.0, 50.0, 12),
    (5, 3, 3.0, 50.0, 12),
    (1, 1, 1.0, 50.0, 16),
    (256, 256, 10.0, 50.0, 20),   # the 4K workload's filter parameters on a small image
]


@pytest.mark.parametrize("H,W,ss,sr,N", CONDITIONED)
def test_plain_forward_matches_oracle(H, W, ss, sr, N):
    f = _image(H, W, seed=H * 1000 + W)
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    out, plan = _gpu_forward(f, ss, sr, N, form="plain", precision="fp32")
    assert plan.info["fit_err"] <= 1e-2
    cond = aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300)
    mask = cond <= 1e4
    assert mask.mean() > 0.99
    err = np.abs(out - ref)[mask].max()
    assert err <= 1e-3, f"max-abs {err}"
    assert plan.diagnostics()["n_guarded"] == aux["n_guard"] == 0


@pytest.mark.parametrize("ss,sr,N", [(3.0, 30.0, 8), (5.0, 25.0, 10), (3.0, 30.0, 12), (2.0, 20.0, 6)])
def test_plain_forward_unconditioned_configs(ss, sr, N):
    f = _image(96, 112, seed=5)
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    out, plan = _gpu_forward(f, ss, sr, N)
    cond = aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300)
    mask = cond <= 1e4
    err = np.abs(out - ref)
    bound = fp32_bound(aux)
    assert np.all(err[mask] <= bound[mask]), f"worst excess {np.max(err[mask] - bound[mask])}"


def test_rects512_exact_and_approximate():
    """512x512 rectangles + noise 10, sigma_s = 3, sigma_r = 30, N = 8: the exact filter on
    the GPU matches the oracle to 1e-3; the approximation (non-convergent at this
    degree) matches the oracle within the FP32 rounding bound; PSNRs are reported."""
    w = synth.workload("rects512")
    f, ss, sr, N = w["f"], w["sigma_s"], w["sigma_r"], w["N"]
    exact_ref = oracle.exact_bf(f, ss, sr)
    ex = bfgc.bf_direct(torch.from_numpy(f).to(DEV), ss, sr)
    torch.cuda.synchronize()
    ex = ex.cpu().numpy().astype(np.float64)
    assert np.abs(ex - exact_ref).max() <= 1e-3
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    out, _ = _gpu_forward(f, ss, sr, N)
    cond = aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300)
    mask = cond <= 1e4
    assert np.all(np.abs(out - ref)[mask] <= fp32_bound(aux)[mask])
    print(f"rects512 PSNR(GPU approx vs exact) = {oracle.psnr_db(out, exact_ref):.2f} dB, "
          f"oracle approx {oracle.psnr_db(ref, exact_ref):.2f} dB")


@pytest.mark.parametrize("H,W,ss,sr", [(97, 131, 2.0, 30.0), (33, 40, 5.0, 10.0), (1, 1, 1.0, 5.0),
                                       (3, 70, 4.0, 50.0), (128, 96, 10.0, 25.0)])
def test_direct_matches_oracle_exact(H, W, ss, sr):
    f = _image(H, W, seed=7)
    ref = oracle.exact_bf(f, ss, sr)
    ex = bfgc.bf_direct(torch.from_numpy(f).to(DEV), ss, sr)
    torch.cuda.synchronize()
    assert np.abs(ex.cpu().numpy() - ref).max() <= 1e-3


def test_constant_image_and_flips():
    out, _ = _gpu_forward(np.full((70, 90), 201.25, dtype=np.float32), 3.0, 50.0, 12)
    assert np.abs(out - 201.25).max() <= 1e-3
    f = _image(80, 100, seed=9)
    a, _ = _gpu_forward(f, 3.0, 50.0, 12)
    b, _ = _gpu_forward(np.ascontiguousarray(f[::-1, ::-1]), 3.0, 50.0, 12)
    assert np.abs(a - b[::-1, ::-1]).max() <= 1e-3


def test_uhd_sampled_outputs_match_oracle():
    """3840x2160 edge + smooth field, sigma_s = 10, sigma_r = 50, N = 20 (the benchmark's
    workload and launch configuration): sampled outputs against the oracle evaluated
    pixel by pixel, corners and borders included."""
    f = synth.workload("uhd")["f"]
    H, W = f.shape
    out, plan = _gpu_forward(f, 10.0, 50.0, 20)
    rng = np.random.default_rng(0)
    ys = np.concatenate([[0, 0, H - 1, H - 1, 1, H - 2, H // 2], rng.integers(0, H, 90)])
    xs = np.concatenate([[0, W - 1, 0, W - 1, W // 2, 3, W - 5], rng.integers(0, W, 90)])
    idx = ys * W + xs
    ref = oracle.gcf_at(f, idx, 10.0, 50.0, 20)
    err = np.abs(out.reshape(-1)[idx] - ref).max()
    assert err <= 1e-3, err


# ----------------------------------------------------------------------------- fused tensor-core form
# Stated tolerance for BF16 channel storage: 0.5 max-abs on [0, 255].  FP16 keeps 3 more
# mantissa bits; on the convergent (sigma_r >= 40) cases it is held to 0.05.
TC_CASES = [c for c in CONDITIONED if c[3] >= 40.0] + [(200, 300, 32.0, 50.0, 12), (150, 170, 20.0, 60.0, 8),
                                                       (130, 150, 4.0, 55.0, 13),    # odd channel count
                                                       (180, 140, 37.0, 50.0, 9),    # a = 7, odd C
                                                       (160, 200, 42.0, 60.0, 8)]    # a = 8: one channel per step


@pytest.mark.parametrize("prec,tol", [("bf16", 0.5), ("fp16", 0.05)])
@pytest.mark.parametrize("H,W,ss,sr,N", TC_CASES)
def test_fused_tc_forward_matches_oracle(H, W, ss, sr, N, prec, tol):
    f = _image(H, W, seed=H * 1000 + W)
    ref, aux = oracle.gcf(f, ss, sr, N, return_pq=True)
    out, plan = _gpu_forward(f, ss, sr, N, form="fused_tc", precision=prec)
    cond = aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300)
    mask = cond <= 1e4
    err = np.abs(out - ref)[mask].max()
    assert err <= tol, f"{prec} max-abs {err}"
    d = plan.diagnostics()
    assert d["n_guarded"] == 0 and d["error_flags"] == 0


def test_fused_tc_fp16_at_paper_operating_point():
    """sigma_r = 30, N = 28 (Table 2): FP16 storage stays within 0.5."""
    f = _image(130, 70, seed=130070)
    ref = oracle.gcf(f, 3.0, 30.0, 28)
    out, _ = _gpu_forward(f, 3.0, 30.0, 28, form="fused_tc", precision="fp16")
    assert np.abs(out - ref).max() <= 0.5


@pytest.mark.xfail(strict=True, reason="BF16 channel storage exceeds the 0.5 bound at sigma_r=30, N=28 "
                                       "(measured 0.67 on this image); FP16 meets it")
def test_fused_tc_bf16_at_paper_operating_point():
    f = _image(130, 70, seed=130070)
    ref = oracle.gcf(f, 3.0, 30.0, 28)
    out, _ = _gpu_forward(f, 3.0, 30.0, 28, form="fused_tc", precision="bf16")
    assert np.abs(out - ref).max() <= 0.5


@pytest.mark.parametrize("prec,tol", [("bf16", 0.5), ("fp16", 0.05)])
def test_fused_tc_uhd_sampled_outputs(prec, tol):
    f = synth.workload("uhd")["f"]
    H, W = f.shape
    out, plan = _gpu_forward(f, 10.0, 50.0, 20, form="fused_tc", precision=prec)
    rng = np.random.default_rng(1)
    ys = np.concatenate([[0, 0, H - 1, H - 1, 1, H - 2, H // 2], rng.integers(0, H, 60)])
    xs = np.concatenate([[0, W - 1, 0, W - 1, W // 2, 3, W - 5], rng.integers(0, W, 60)])
    idx = ys * W + xs
    ref = oracle.gcf_at(f, idx, 10.0, 50.0, 20)
    assert np.abs(out.reshape(-1)[idx] - ref).max() <= tol


def test_fused_tc_matches_plain_on_constant_and_flips():
    out, _ = _gpu_forward(np.full((70, 90), 201.25, dtype=np.float32), 3.0, 50.0, 12, form="fused_tc",
                          precision="fp16")
    assert np.abs(out - 201.25).max() <= 0.05
    f = _image(80, 100, seed=9)
    a, _ = _gpu_forward(f, 3.0, 50.0, 12, form="fused_tc", precision="fp16")
    b, _ = _gpu_forward(np.ascontiguousarray(f[::-1, ::-1]), 3.0, 50.0, 12, form="fused_tc", precision="fp16")
    assert np.abs(a - b[::-1, ::-1]).max() <= 0.05


# ----------------------------------------------------------------------------- recursive form
@pytest.mark.parametrize("H,W,ss,sr,N", [(97, 131, 2.0, 50.0, 12), (64, 200, 5.0, 60.0, 10),
                                         (40, 33, 10.0, 50.0, 16), (1, 37, 2.0, 50.0, 12),
                                         (5, 3, 3.0, 50.0, 12), (150, 170, 20.0, 60.0, 8),
                                         (96, 96, 0.7, 50.0, 12),
                                         # rows split into three segments each (warm-up joins)
                                         (700, 650, 2.0, 50.0, 12), (520, 530, 4.0, 50.0, 10)])
def test_recursive_forward_matches_oracle_twin(H, W, ss, sr, N):
    """Young-van Vliet recursive spatial filter: FP32 GPU against the FP64 oracle running
    the same recursion, padding and initialisation."""
    f = _image(H, W, seed=H * 7 + W)
    ref, aux = oracle.gcf(f, ss, sr, N, spatial="recursive", return_pq=True)
    out, plan = _gpu_forward(f, ss, sr, N, form="recursive")
    cond = aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300)
    mask = cond <= 1e4
    assert np.abs(out - ref)[mask].max() <= 1e-3
    exact = oracle.exact_bf(f, ss, sr)
    print(f"recursive {H}x{W} sigma_s={ss}: PSNR vs exact {oracle.psnr_db(out, exact):.1f} dB "
          f"(direct form {oracle.psnr_db(oracle.gcf(f, ss, sr, N), exact):.1f} dB)")


def test_recursive_form_has_no_backward():
    f = torch.from_numpy(_image(32, 32, seed=1)).cuda()
    plan = api.GCPlan(32, 32, 2.0, 50.0, 8, form="recursive")
    with pytest.raises(bfgc.BfError) as e:
        plan.backward(f, torch.ones_like(f))
    assert e.value.status == bfgc.BF_ERR_UNSUPPORTED
