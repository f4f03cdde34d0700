"""Row strips of one image (paper_1605_02178_gb300/strips.py) through the C ABI on one GPU:
the ranks are emulated in one process (each strip's halo rows are sliced from the image, as
the exchange would deliver them), and the strips put together are compared with the
whole-image call.

The plain and fused FP32 forms take per pixel the same operations on the same rows whether
the image is whole or cut, so their strips are equal bit for bit.  The tensor-core form's
column pass groups the band's products in tiles that start at another row in a strip, which
changes the FP32 summation order only (held to 0.05 max-abs; its parity bound against the
FP64 oracle is 0.5).  The adjoint (plain kernels) is compared to 1e-5 of the gradient's
scale, dL/dsigma_r (a sum of per-strip FP64 reductions) to 1e-6 relative."""
import numpy as np
import pytest
import torch

from paper_1605_02178_gb300 import api, strips, synth

pytestmark = pytest.mark.gpu

DEV = "cuda"


def _emulated_forward(f, world, ss, sr, N, **opts):
    H = f.shape[0]
    R = strips.window_radius(ss)
    parts = []
    for k in range(world):
        y0, y1 = strips.strip_rows(H, world, k)
        e0, e1 = strips.halo_range(H, y0, y1, R)
        parts.append(strips.forward_strip(f[e0:e1], (e0, e1), (y0, y1), ss, sr, N, **opts))
    return torch.cat(parts)


@pytest.mark.parametrize("world", [2, 3, 8])
@pytest.mark.parametrize("H,W,ss,sr,N", [(300, 517, 10.0, 50.0, 20), (97, 131, 2.0, 40.0, 12)])
@pytest.mark.parametrize("form,precision", [("plain", "fp32"), ("fused", "fp32"), ("fused_tc", "bf16")])
def test_strips_equal_the_whole_image(world, H, W, ss, sr, N, form, precision):
    f = torch.from_numpy(synth.edge_smooth_image(H, W, noise_std=5.0, seed=H + W)).to(DEV)
    whole = api.GCPlan(H, W, ss, sr, N, form=form, precision=precision).forward(f)
    cut = _emulated_forward(f, world, ss, sr, N, form=form, precision=precision)
    torch.cuda.synchronize()
    if precision == "fp32":
        assert torch.equal(cut, whole)
    else:
        assert (cut - whole).abs().max().item() <= 0.05


def test_strips_refuse_the_recursive_form():
    f = torch.zeros(64, 64, device=DEV)
    with pytest.raises(ValueError):
        strips.forward_strip(f, (0, 64), (0, 32), 3.0, 40.0, 8, form="recursive")


@pytest.mark.parametrize("world", [2, 5])
def test_strip_adjoint_equals_the_whole_image(world):
    H, W, ss, sr, N = 150, 170, 3.0, 40.0, 10
    f = torch.from_numpy(synth.edge_smooth_image(H, W, seed=7)).to(DEV)
    w = torch.from_numpy(np.random.default_rng(8).standard_normal((H, W)).astype(np.float32)).to(DEV)
    gf_ref, gs_ref = api.GCPlan(H, W, ss, sr, N).backward(f, w)
    R = strips.window_radius(ss)
    parts, gs = [], 0.0
    for k in range(world):
        y0, y1 = strips.strip_rows(H, world, k)
        e0, e1 = strips.halo_range(H, y0, y1, 2 * R)
        a0, a1 = strips.halo_range(H, y0, y1, R)
        g, s = strips.backward_strip(f[e0:e1], w[a0:a1], H, (y0, y1), ss, sr, N)
        parts.append(g)
        gs += float(s)
    gf = torch.cat(parts)
    torch.cuda.synchronize()
    scale = gf_ref.abs().max().item()
    assert (gf - gf_ref).abs().max().item() <= 1e-5 * scale
    assert abs(gs - float(gs_ref)) <= 1e-6 * abs(float(gs_ref))
