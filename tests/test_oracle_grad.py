"""Pins for the gradient oracle (oracle.grad_ref): its forward equals the C oracle,
and its autograd gradients equal central finite differences of the C oracle."""
import numpy as np
import pytest
import torch

import oracle
from oracle import grad_ref
from paper_1605_02178_gb300 import synth


@pytest.mark.parametrize("ss,sr,N", [(1.5, 50.0, 12), (2.0, 30.0, 8), (1.0, 25.0, 10)])
def test_torch_forward_equals_c_oracle(ss, sr, N):
    f = synth.rects_image(21, 26, n_rects=5, noise_std=10.0, seed=11).astype(np.float64)
    ref = oracle.gcf(f, ss, sr, N)
    out = grad_ref.gcf_t(torch.tensor(f), ss, torch.tensor(sr, dtype=torch.float64), N)
    assert np.allclose(out.numpy(), ref, rtol=0, atol=1e-9)


@pytest.mark.parametrize("ss,sr,N", [(1.0, 50.0, 12), (1.5, 40.0, 10)])
def test_gradients_match_central_differences(ss, sr, N):
    f = synth.rects_image(12, 14, n_rects=3, noise_std=10.0, seed=12).astype(np.float64)
    w = synth.weight_map(12, 14, seed=13).astype(np.float64)
    _, gf, gs = grad_ref.loss_and_grads(f, w, ss, sr, N)
    loss = lambda img, s: float((w * oracle.gcf(img, ss, s, N)).sum())
    h = 1e-3
    rng = np.random.default_rng(0)
    for p in rng.choice(f.size, size=40, replace=False):
        fp, fm = f.copy().reshape(-1), f.copy().reshape(-1)
        fp[p] += h
        fm[p] -= h
        fd = (loss(fp.reshape(f.shape), sr) - loss(fm.reshape(f.shape), sr)) / (2 * h)
        assert gf.reshape(-1)[p] == pytest.approx(fd, rel=1e-5, abs=1e-8), p
    hs = 1e-4 * sr
    fd = (loss(f, sr + hs) - loss(f, sr - hs)) / (2 * hs)
    assert gs == pytest.approx(fd, rel=1e-5, abs=1e-8)
