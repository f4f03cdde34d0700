"""bf_gc_forward_host_stream: streaming forward of images held in host memory (uploads,
filtering and downloads of consecutive images overlapped).  Host-side argument checks run on
the CPU (they precede every CUDA call); on the GPU every image must equal the per-image
forward of the same plan bit for bit, for pinned and pageable host buffers."""
import ctypes

import numpy as np
import pytest
import torch

from paper_1605_02178_gb300 import api, bfgc as B, synth


def test_stream_bytes_cover_two_slots_and_a_workspace():
    plan = api.GCPlan(100, 130, 3.0, 40.0, 8, form="fused_tc", precision="bf16")
    fwd = plan.workspace_bytes()[0]
    img = -(-100 * 130 * 4 // 256) * 256
    assert B.bf_gc_stream_bytes(plan.handle) == 4 * img + -(-fwd // 256) * 256


def test_stream_rejects_bad_arguments_before_any_cuda_call():
    plan = api.GCPlan(16, 16, 2.0, 40.0, 4)
    L = B.lib()
    arr = (ctypes.c_void_p * 2)(16, 32)
    nul = (ctypes.c_void_p * 2)(16, None)
    need = B.bf_gc_stream_bytes(plan.handle)
    assert L.bf_gc_forward_host_stream(plan.handle, 0, arr, arr, ctypes.c_void_p(256), need, None) == B.BF_ERR_INVALID_ARG
    assert L.bf_gc_forward_host_stream(plan.handle, 2, nul, arr, ctypes.c_void_p(256), need, None) == B.BF_ERR_INVALID_ARG
    assert L.bf_gc_forward_host_stream(plan.handle, 2, arr, arr, ctypes.c_void_p(256), need - 1, None) == B.BF_ERR_WORKSPACE
    assert L.bf_gc_forward_host_stream(plan.handle, 2, arr, arr, ctypes.c_void_p(264), need, None) == B.BF_ERR_WORKSPACE


@pytest.mark.gpu
@pytest.mark.parametrize("form,precision", [("fused_tc", "bf16"), ("plain", "fp32")])
@pytest.mark.parametrize("count,pinned", [(1, True), (2, True), (5, True), (7, False)])
def test_stream_equals_per_image_forwards(form, precision, count, pinned):
    H, W = 257, 301
    plan = api.GCPlan(H, W, 6.0, 50.0, 12, form=form, precision=precision)
    imgs = [torch.from_numpy(synth.edge_smooth_image(H, W, seed=40 + i)) for i in range(count)]
    if pinned:
        imgs = [t.pin_memory() for t in imgs]
    outs = [torch.full_like(t, -1.0) for t in imgs]
    if pinned:
        outs = [t.pin_memory() for t in outs]
    scratch = torch.empty(B.bf_gc_stream_bytes(plan.handle), dtype=torch.uint8, device="cuda")
    B.bf_gc_forward_host_stream(plan.handle, imgs, outs, scratch)
    for t, o in zip(imgs, outs):
        ref = plan.forward(t.cuda()).cpu()
        assert torch.equal(o, ref)
