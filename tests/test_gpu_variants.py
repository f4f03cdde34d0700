"""GPU tests of the Gauss-polynomial variant (c_n = 1/n!, the Gauss-polynomial filter recalled
in Sec. II), of the Table 1 comparison between the two polynomial families run on the GPU,
and of the FP16 / BF16 channel-storage study over the window sizes of the 8192x8192 sweep
(at a reduced image size).

Tolerances are those of the forward tests: FP32 within the first-order rounding bound of P/Q
(plus 1e-3), BF16 0.5 and FP16 0.05 max-abs on conditioned pixels (sum|terms of Q|/|Q| <= 1e4).
"""
import json
import os

import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, bfgc, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _gpu_forward(f, ss, sr, N, **opts):
    plan = api.GCPlan(f.shape[0], f.shape[1], ss, sr, N, **opts)
    out = plan.forward(torch.from_numpy(f).to(DEV))
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.float64), plan


def _cond_mask(aux):
    return aux["Qabs"] / np.maximum(np.abs(aux["Q"]), 1e-300) <= 1e4


def _fp32_bound(aux, eps=4e-6):
    Q = np.maximum(np.abs(aux["Q"]), 1e-300)
    return eps * (aux["Pabs"] + np.abs(aux["P"]) / Q * aux["Qabs"]) / Q + 1e-3


GPF_CASES = [(97, 131, 2.0, 80.0, 12), (256, 256, 5.0, 60.0, 16), (130, 70, 10.0, 100.0, 8)]


@pytest.mark.parametrize("form,prec,tol", [("plain", "fp32", None), ("fused_tc", "fp16", 0.05),
                                           ("fused_tc", "bf16", 0.5), ("recursive", "fp32", None)])
@pytest.mark.parametrize("H,W,ss,sr,N", GPF_CASES)
def test_gpf_variant_matches_oracle(H, W, ss, sr, N, form, prec, tol):
    """The GPU forms with c_n = 1/n! against the oracle run with the same coefficients."""
    f = synth.rects_image(H, W, n_rects=8, noise_std=10.0, seed=H + W)
    spatial = "recursive" if form == "recursive" else "separable"
    ref, aux = oracle.gcf(f, ss, sr, N, c=oracle.taylor_coeffs(N), spatial=spatial, return_pq=True)
    out, plan = _gpu_forward(f, ss, sr, N, form=form, precision=prec, poly="taylor")
    assert np.allclose(plan.info["c"][: N + 1], oracle.taylor_coeffs(N), rtol=1e-12)
    mask = _cond_mask(aux)
    assert mask.mean() > 0.99
    err = np.abs(out - ref)[mask]
    if tol is None:
        assert np.all(err <= _fp32_bound(aux)[mask]), err.max()
    else:
        assert err.max() <= tol, err.max()
    assert plan.diagnostics()["error_flags"] == 0


def test_table1_gpf_vs_gcf_on_gpu():
    """Table 1 (Sec. IV) run on the GPU: MSE in dB of the Gauss-polynomial and the
    Gauss-Chebyshev filters against the exact filter (the GPU's bf_direct) on the synthetic
    150x150 checkerboard, sigma_s = 5, sigma_r = 30.  The GPU result of each filter deviates
    from the FP64 oracle's by at least 10 dB less than the oracle's own approximation error
    (or lies below -60 dB), the GPF row stays within 2 dB of the printed values and the GCF
    row is more than 10 dB below it at every degree."""
    g = json.load(open(os.path.join(GOLDEN, "table1_checker_mse_db.json")))
    ss, sr = g["sigma_s"], g["sigma_r"]
    f = synth.checkerboard()
    ex_gpu = bfgc.bf_direct(torch.from_numpy(f).to(DEV), ss, sr)
    torch.cuda.synchronize()
    ex = ex_gpu.cpu().numpy().astype(np.float64)
    ex_ref = oracle.exact_bf(f, ss, sr)
    assert np.abs(ex - ex_ref).max() <= 1e-3
    for N, gpf_ref, _ in zip(g["N"], g["GPF"], g["GCF"]):
        gpf_gpu, _ = _gpu_forward(f, ss, sr, N, form="plain", poly="taylor")
        gcf_gpu, _ = _gpu_forward(f, ss, sr, N, form="plain")
        gpf_or = oracle.gcf(f, ss, sr, N, c=oracle.taylor_coeffs(N))
        gcf_or = oracle.gcf(f, ss, sr, N)
        for gpu, orc in ((gpf_gpu, gpf_or), (gcf_gpu, gcf_or)):
            dev_db = oracle.mse_db(gpu, orc)
            assert dev_db < max(oracle.mse_db(orc, ex_ref) - 10.0, -60.0), (N, dev_db)
        gpf_db, gcf_db = oracle.mse_db(gpf_gpu, ex), oracle.mse_db(gcf_gpu, ex)
        assert abs(gpf_db - gpf_ref) < 2.0, (N, gpf_db, gpf_ref)
        assert gcf_db < gpf_db - 10.0, (N, gcf_db, gpf_db)


def test_gpf_vs_gcf_at_4k_on_gpu():
    """The same comparison at full scale, on the 3840x2160 continuous-tone benchmark image
    (sigma_s = 5, sigma_r = 30; GPU FP32, exact filter from bf_direct): here the ordering of
    Table 1 reverses.  On the binary checkerboard every range product t tau / sigma_r^2 of
    the kernel sits at +-mu, where the Chebyshev interpolant's equi-oscillating error beats
    the Taylor polynomial's; on a continuous-tone image the products gather near 0, where the
    Taylor polynomial is nearly exact, and the fixed interval [-mu, mu] (mu = 18 at
    sigma_r = 30) needs N of about 28 before the Chebyshev fit converges.  The GPU values
    follow the FP64 oracle on a 160-row strip (checked on the CPU when this test was written:
    GPF 5.3 / -31.9 / -80.5 dB, GCF 90.7 / 74.9 / 75.0 dB at N = 4 / 12 / 20)."""
    f = synth.workload("uhd")["f"]
    ft = torch.from_numpy(f).to(DEV)
    ex = bfgc.bf_direct(ft, 5.0, 30.0)
    torch.cuda.synchronize()
    exn = ex.cpu().numpy().astype(np.float64)
    last_gpf = np.inf
    for N in (4, 8, 12, 16, 20, 25):
        outs = {}
        for poly in ("taylor", "chebyshev"):
            plan = api.GCPlan(2160, 3840, 5.0, 30.0, N, form="plain", poly=poly)
            outs[poly] = plan.forward(ft).cpu().numpy().astype(np.float64)
        gpf_db, gcf_db = oracle.mse_db(outs["taylor"], exn), oracle.mse_db(outs["chebyshev"], exn)
        assert gpf_db < gcf_db - 20.0, (N, gpf_db, gcf_db)
        assert gpf_db < last_gpf, (N, gpf_db, last_gpf)
        last_gpf = gpf_db


# ---------------------------------------------------------------- precision study (reduced cfg4)
@pytest.mark.parametrize("ss", [8.0, 16.0, 32.0])
@pytest.mark.parametrize("N", [12, 28])
def test_precision_study_reduced(ss, N):
    """Channel storage precision over the window sizes of the 8192x8192 sweep, at 768x768:
    FP16 and BF16 (fused tensor-core form) and FP32 (plain) against the FP64 oracle at
    sigma_r = 30.  N = 28 (fit converged): on conditioned pixels FP32 within its rounding
    bound, FP16 (channels stored times 2^14) below 0.05 max-abs and at least 4x below BF16
    in RMS, BF16 within 0.5.  N = 12 (fit error 2e4: the approximation itself is
    meaningless there, and its huge alternating coefficients amplify rounding inside the
    filtered channels beyond what sum|terms of Q| / |Q| measures; parity unpinned): every
    form finishes without flags and with finite outputs."""
    f = synth.edge_smooth_image(768, 768, noise_std=5.0, seed=5)
    ref, aux = oracle.gcf(f, ss, 30.0, N, return_pq=True)
    mask = _cond_mask(aux)
    res = {}
    for form, prec in (("plain", "fp32"), ("fused_tc", "fp16"), ("fused_tc", "bf16")):
        out, plan = _gpu_forward(f, ss, 30.0, N, form=form, precision=prec)
        assert plan.diagnostics()["error_flags"] == 0
        assert np.isfinite(out).all()
        res[prec] = np.abs(out - ref)[mask]
    if N == 28:
        assert np.all(res["fp32"] <= _fp32_bound(aux)[mask])
        rms = {k: float(np.sqrt(np.mean(v ** 2))) for k, v in res.items()}
        assert res["fp16"].max() <= 0.05, res["fp16"].max()
        assert rms["fp16"] * 4.0 <= rms["bf16"], rms
        assert res["bf16"].max() <= 0.5, res["bf16"].max()
