"""bf_gc_forward_static: the forward for callers that cannot allocate device memory when
they filter (plug-ins whose host application owns the allocator, real-time pipelines
that forbid cudaMalloc after start-up).  It keeps its scratch in a fixed device array
inside the library instead of a caller workspace.

Checked through the C ABI against the workspace entry point bf_gc_forward on two
calls in a row (the second call must not see the first call's leftovers), with the
FP32 forward tolerance used elsewhere (1e-3 max-abs on [0, 255]).  This file sorts
last so that a run stopping at the first failure has run every other test.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1605_02178_gb300 import bfgc as B, synth

pytestmark = pytest.mark.gpu


def test_static_scratch_forward_matches_workspace_forward():
    H, W, ss, sr, N = 300, 257, 3.0, 50.0, 12
    plan = B.bf_gc_plan(H, W, ss, sr, N)
    try:
        fwd_bytes, _ = B.bf_gc_workspace_size(plan)
        assert fwd_bytes <= B.BF_STATIC_SCRATCH_BYTES
        ws = torch.empty(fwd_bytes, dtype=torch.uint8, device="cuda")
        stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        for seed in (11, 12):                       # two calls in a row, different images
            f = torch.from_numpy(synth.rects_image(H, W, n_rects=8, seed=seed)).cuda()
            ref = torch.empty_like(f)
            out = torch.full_like(f, float("nan"))
            B.bf_gc_forward(plan, f, ref, ws)
            st = B.lib().bf_gc_forward_static(plan, ctypes.c_void_p(f.data_ptr()),
                                              ctypes.c_void_p(out.data_ptr()), stream)
            assert st == B.BF_OK, B.bf_status_string(st)
            torch.cuda.synchronize()
            err = float((out - ref).abs().max())
            assert np.isfinite(err) and err <= 1e-3, err
    finally:
        B.bf_gc_plan_destroy(plan)


def test_static_scratch_rejects_plans_beyond_its_size():
    plan = B.bf_gc_plan(2160, 3840, 10.0, 50.0, 20)
    try:
        assert B.bf_gc_workspace_size(plan)[0] > B.BF_STATIC_SCRATCH_BYTES
        f = torch.zeros(2160, 3840, device="cuda")
        out = torch.empty_like(f)
        st = B.lib().bf_gc_forward_static(plan, ctypes.c_void_p(f.data_ptr()),
                                          ctypes.c_void_p(out.data_ptr()), None)
        assert st == B.BF_ERR_WORKSPACE
    finally:
        B.bf_gc_plan_destroy(plan)
