"""GPU adjoint (bf_gc_backward) against the gradient oracle (float64 autograd of the
same approximation, itself pinned to central finite differences of the C oracle).

Tolerance: FP32 gradients, max-abs error <= 2e-3 * max |reference gradient| for dL/df
and relative error <= 2e-3 for dL/dsigma_r, on convergent configurations.
"""
import numpy as np
import pytest
import torch

import oracle
from oracle import grad_ref
from paper_1605_02178_gb300 import api, bfgc, synth

pytestmark = pytest.mark.gpu


def _gpu_grads(f, w, ss, sr, N, form="plain", precision="fp32", save=False):
    plan = api.GCPlan(f.shape[0], f.shape[1], ss, sr, N, form=form, precision=precision, save_channels=save)
    ft = torch.from_numpy(f).cuda()
    wt = torch.from_numpy(w).cuda()
    if save:
        ws = plan.workspace("bwd")
        plan.forward(ft, ws=ws)
        gf, gs = plan.backward(ft, wt, ws=ws)
    else:
        gf, gs = plan.backward(ft, wt)
    torch.cuda.synchronize()
    return gf.cpu().numpy().astype(np.float64), float(gs.item())


CASES = [
    (40, 52, 2.0, 50.0, 12),
    (64, 64, 3.0, 40.0, 16),
    (33, 17, 5.0, 60.0, 10),      # window wider than the image on one axis
    (7, 9, 4.0, 50.0, 12),        # repeated reflection on both axes
    (1, 30, 2.0, 50.0, 8),
    (96, 80, 5.0, 50.0, 20),
    (150, 530, 8.0, 50.0, 12),    # several row and column blocks, fold-back at all four edges
]


@pytest.mark.parametrize("H,W,ss,sr,N", CASES)
def test_backward_matches_gradient_oracle(H, W, ss, sr, N):
    f = synth.rects_image(H, W, n_rects=6, noise_std=10.0, seed=H + W)
    w = synth.weight_map(H, W, seed=H * W)
    _, gref, sref = grad_ref.loss_and_grads(f, w, ss, sr, N)
    gf, gs = _gpu_grads(f, w, ss, sr, N)
    scale = np.abs(gref).max()
    assert np.abs(gf - gref).max() <= 2e-3 * scale, np.abs(gf - gref).max() / scale
    assert gs == pytest.approx(sref, rel=2e-3, abs=1e-6 * scale)


def test_backward_with_saved_channels_equals_recompute():
    f = synth.rects_image(70, 90, seed=3)
    w = synth.weight_map(70, 90, seed=4)
    a, sa = _gpu_grads(f, w, 3.0, 50.0, 12)
    b, sb = _gpu_grads(f, w, 3.0, 50.0, 12, save=True)
    assert np.array_equal(a, b) and sa == sb


def test_backward_after_fused_forward_form():
    """The backward of a fused-form plan is the FP32 adjoint of the same approximation."""
    f = synth.rects_image(48, 64, seed=5)
    w = synth.weight_map(48, 64, seed=6)
    _, gref, sref = grad_ref.loss_and_grads(f, w, 2.0, 50.0, 12)
    gf, gs = _gpu_grads(f, w, 2.0, 50.0, 12, form="fused_tc", precision="bf16")
    assert np.abs(gf - gref).max() <= 2e-3 * np.abs(gref).max()
    assert gs == pytest.approx(sref, rel=2e-3)


def test_autograd_function():
    f = synth.rects_image(50, 60, seed=7)
    w = synth.weight_map(50, 60, seed=8)
    _, gref, sref = grad_ref.loss_and_grads(f, w, 2.0, 50.0, 12)
    plan = api.GCPlan(50, 60, 2.0, 50.0, 12)
    ft = torch.from_numpy(f).cuda().requires_grad_(True)
    st = torch.tensor(50.0, device="cuda", requires_grad=True)
    out = api.GCBilateral.apply(ft, st, plan)
    (torch.from_numpy(w).cuda() * out).sum().backward()
    g = ft.grad.cpu().numpy().astype(np.float64)
    assert np.abs(g - gref).max() <= 2e-3 * np.abs(gref).max()
    assert float(st.grad) == pytest.approx(sref, rel=2e-3)


def test_grad1024_crop_against_oracle_and_finite_differences():
    """1024x1024 rectangles + noise 20, loss = sum(w * B[f]), sigma_s = 5; the gradient on a
    seeded 64x64 crop against the oracle gradient, at the non-convergent pair
    (sigma_r = 25, N = 10) and at the convergent anchor (sigma_r = 50, N = 12)."""
    wl = synth.workload("grad1024")
    f, w = wl["f"], wl["w"]
    rng = np.random.default_rng(0)
    y0, x0 = (int(v) for v in rng.integers(64, 1024 - 128, 2))     # interior: FD windows fit
    for sr, N, tol in ((50.0, 12, 2e-3), (25.0, 10, None)):
        _, gref, sref = grad_ref.loss_and_grads(f, w, 5.0, sr, N)
        gf, gs = _gpu_grads(f, w, 5.0, sr, N)
        crop = (slice(y0, y0 + 64), slice(x0, x0 + 64))
        err = np.abs(gf[crop] - gref[crop]).max() / np.abs(gref[crop]).max()
        if tol is None:
            print(f"sigma_r={sr}, N={N} (non-convergent): crop rel err {err:.3e}, "
                  f"dsigma {gs:.6e} vs {sref:.6e}")
            assert np.isfinite(err)
        else:
            assert err <= tol, err
            assert gs == pytest.approx(sref, rel=tol)
    # central differences of the FP64 oracle at a few crop pixels (convergent anchor)
    _, gref, _ = grad_ref.loss_and_grads(f, w, 5.0, 50.0, 12)
    R = oracle.window_radius(5.0)
    for k in range(4):
        yy, xx = y0 + 8 + 13 * k, x0 + 5 + 11 * k
        ys, xs = slice(yy - 2 * R, yy + 2 * R + 1), slice(xx - 2 * R, xx + 2 * R + 1)
        sub, wsub = f[ys, xs].astype(np.float64), w[ys, xs].astype(np.float64)
        inner = (slice(R, 3 * R + 1), slice(R, 3 * R + 1))
        h = 1e-3

        def loss(img):
            return float((wsub[inner] * oracle.gcf(img, 5.0, 50.0, 12)[inner]).sum())
        fp, fm = sub.copy(), sub.copy()
        fp[2 * R, 2 * R] += h
        fm[2 * R, 2 * R] -= h
        fd = (loss(fp) - loss(fm)) / (2 * h)
        assert gref[yy, xx] == pytest.approx(fd, rel=1e-5, abs=1e-9)


@pytest.mark.parametrize("dtype", [torch.float64, torch.float32])
def test_autograd_function_with_saved_channels(dtype):
    """GCBilateral on a save_channels plan: the backward reuses the channels of its own forward
    (a workspace kept per call), giving the recomputing plan's gradients bit for bit; dL/dsigma_r
    comes back in sigma_r's dtype and shape; a sigma_r other than the plan's is refused."""
    H, W, ss, sr, N = 70, 90, 3.0, 50.0, 12
    f = torch.from_numpy(synth.rects_image(H, W, seed=3)).cuda()
    w = torch.from_numpy(synth.weight_map(H, W, seed=4)).cuda()
    grads = []
    for save in (False, True):
        plan = api.GCPlan(H, W, ss, sr, N, save_channels=save)
        x = f.clone().requires_grad_(True)
        s_r = torch.tensor(sr, dtype=dtype, device="cuda", requires_grad=True)
        other = torch.from_numpy(synth.rects_image(H, W, seed=5)).cuda()
        out = api.GCBilateral.apply(x, s_r, plan)
        plan.forward(other)                       # another image through the same plan in between
        (out * w).sum().backward()
        torch.cuda.synchronize()
        assert s_r.grad.dtype == dtype and s_r.grad.shape == s_r.shape
        grads.append((x.grad.clone(), float(s_r.grad)))
    assert torch.equal(grads[0][0], grads[1][0]) and grads[0][1] == grads[1][1]
    with pytest.raises(ValueError):
        api.GCBilateral.apply(f.clone().requires_grad_(True), torch.tensor(sr + 1.0, device="cuda"),
                              api.GCPlan(H, W, ss, sr, N))
