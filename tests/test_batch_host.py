"""CPU checks of the batch host logic (bf_gc_batch_create / _workspace_size / _info: no CUDA
call), of the row-pass tile-width option, and of the autotuner's choices and JSON cache
(with a fake timer).  No kernel is launched here."""
import json

import numpy as np
import pytest

from paper_1605_02178_gb300 import autotune, bfgc as B, synth
from paper_1605_02178_gb300.api import GCPlan


def _plans(specs, form="fused_tc", precision="bf16"):
    return [GCPlan(s["H"], s["W"], s["sigma_s"], s["sigma_r"], s["N"], form=form, precision=precision)
            for s in specs]


def _cost(plan):
    """Cost model of the branch split (the tensor-core form's banded products per pixel)."""
    i = plan.info
    return plan.H * plan.W * i["C"] * (128.0 + 32.0 * np.ceil(i["R"] / 16.0))


@pytest.mark.parametrize("k", [1, 3, 8, 64])
def test_batch_split_covers_every_image_and_balances(k):
    specs = synth.batch_specs(40, seed=4)
    plans = _plans(specs)
    h = B.bf_gc_batch_create([p.handle for p in plans], k)
    try:
        br, captures = B.bf_gc_batch_info(h, len(plans))
        assert captures == 0
        kk = min(k, len(plans))
        assert set(br) <= set(range(kk)) and len(br) == len(plans)
        if kk <= len(plans):
            assert len(set(br)) == kk                  # no branch left empty
        cost = np.array([_cost(p) for p in plans])
        load = np.array([cost[np.array(br) == j].sum() for j in range(kk)])
        # longest-processing-time-first bound: no branch exceeds the mean by more than one image
        assert load.max() <= load.mean() + cost.max() + 1e-6
        # workspace: per branch, the largest forward workspace among its images
        need = sum(max(-(-B.bf_gc_workspace_size(plans[i].handle)[0] // 256) * 256
                       for i in range(len(plans)) if br[i] == j) for j in range(kk))
        assert B.bf_gc_batch_workspace_size(h) == need
    finally:
        B.bf_gc_batch_destroy(h)


def test_batch_create_rejects_bad_arguments():
    plans = _plans(synth.batch_specs(3, seed=4))
    handles = [p.handle for p in plans]
    for branches in (0, 65):
        with pytest.raises(B.BfError) as e:
            B.bf_gc_batch_create(handles, branches)
        assert e.value.status == B.BF_ERR_INVALID_ARG
    with pytest.raises(B.BfError) as e:
        B.bf_gc_batch_create([], 2)
    assert e.value.status == B.BF_ERR_INVALID_ARG
    with pytest.raises(B.BfError) as e:
        B.bf_gc_batch_create(handles[:1] + [None], 2)
    assert e.value.status == B.BF_ERR_INVALID_ARG
    B.bf_gc_profile_enable(plans[0].handle, True)
    with pytest.raises(B.BfError) as e:
        B.bf_gc_batch_create(handles, 2)
    assert e.value.status == B.BF_ERR_INVALID_ARG


def test_batch_forward_rejects_bad_workspace_before_any_cuda_call():
    plans = _plans(synth.batch_specs(2, seed=4))
    h = B.bf_gc_batch_create([p.handle for p in plans], 2)
    try:
        import ctypes
        arr = (ctypes.c_void_p * 2)(16, 32)
        st = B.lib().bf_gc_batch_forward(h, arr, arr, None, 0, None)
        assert st == B.BF_ERR_WORKSPACE
        st = B.lib().bf_gc_batch_forward(h, arr, arr, ctypes.c_void_p(256 + 8), 1 << 40, None)
        assert st == B.BF_ERR_WORKSPACE
        nul = (ctypes.c_void_p * 2)(16, None)
        st = B.lib().bf_gc_batch_forward(h, nul, arr, ctypes.c_void_p(256), 1 << 40, None)
        assert st == B.BF_ERR_INVALID_ARG
        # inputs and outputs start on 16-byte boundaries
        for bad_f, bad_o in (((16, 36), (16, 32)), ((16, 32), (24, 32))):
            pf, po = (ctypes.c_void_p * 2)(*bad_f), (ctypes.c_void_p * 2)(*bad_o)
            st = B.lib().bf_gc_batch_forward(h, pf, po, ctypes.c_void_p(256), 1 << 40, None)
            assert st == B.BF_ERR_INVALID_ARG
    finally:
        B.bf_gc_batch_destroy(h)


def test_tile_width_option():
    p = B.bf_gc_plan(100, 100, 10.0, 30.0, 8)           # R = 30, a = 2
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_FORM, B.BF_FORM_FUSED_TC)
        for tw in (0, 64, 128, 256):
            B.bf_gc_plan_set(p, B.BF_OPT_TILE_W, tw)
        for bad in (32, 96, 512, 1.5, -64):
            with pytest.raises(B.BfError) as e:
                B.bf_gc_plan_set(p, B.BF_OPT_TILE_W, bad)
            assert e.value.status == B.BF_ERR_INVALID_ARG
    finally:
        B.bf_gc_plan_destroy(p)
    p = B.bf_gc_plan(100, 100, 25.0, 30.0, 8)           # R = 75, a = 5: 64 only
    try:
        B.bf_gc_plan_set(p, B.BF_OPT_TILE_W, 64)
        for tw in (128, 256):
            with pytest.raises(B.BfError) as e:
                B.bf_gc_plan_set(p, B.BF_OPT_TILE_W, tw)
            assert e.value.status == B.BF_ERR_UNSUPPORTED
    finally:
        B.bf_gc_plan_destroy(p)


def test_tile_width_leaves_workspace_unchanged():
    a = GCPlan(333, 517, 5.0, 30.0, 10, form="fused_tc", precision="bf16")
    b = GCPlan(333, 517, 5.0, 30.0, 10, form="fused_tc", precision="bf16", tile_w=64)
    assert a.workspace_bytes() == b.workspace_bytes()


def test_autotuner_picks_fastest_and_caches(tmp_path):
    path = tmp_path / "tune.json"
    calls = []

    def fake(kind, **kw):
        calls.append((kind, kw["tile_w"]))
        return {0: 1.5, 64: 3.0, 128: 1.0, 256: 2.0}[kw["tile_w"]]

    t = autotune.Autotuner(path=str(path), device_name="fake-gpu", measure=fake)
    assert t.tile_w(30, 10, 1000, "bf16") == 128
    assert len(calls) == 4
    assert t.tile_w(30, 10, 900, "bf16") == 128          # same bucket: cached, no new timing
    assert len(calls) == 4
    assert t.tile_w(90, 10, 900, "bf16") == 0            # a = 6: only kernels 0 and 64 exist
    assert len(calls) == 6 and {c[1] for c in calls[4:]} == {0, 64}
    t.tile_w(30, 10, 100, "bf16")                        # another width class
    assert len(calls) == 10
    assert t.branches("sig", lambda k: {1: 9, 2: 5, 4: 3, 8: 3, 16: 4}[k]) == 4   # ties: fewer branches
    data = json.loads(path.read_text())
    assert data["fake-gpu"]["tile_w"][autotune.tile_bucket(30, 10, 1000, "bf16")] == 128
    assert data["fake-gpu"]["branches"]["sig"] == 4
    # a new tuner reads the cache and measures nothing
    t2 = autotune.Autotuner(path=str(path), device_name="fake-gpu",
                            measure=lambda *a, **k: pytest.fail("measured a cached bucket"))
    assert t2.tile_w(30, 10, 1000, "bf16") == 128
    assert t2.branches("sig", lambda k: pytest.fail("timed a cached batch")) == 4
    # another device name has its own entries
    t3 = autotune.Autotuner(path=str(path), device_name="other", measure=lambda kind, **kw: 1.0 / (1 + kw["tile_w"]))
    assert t3.tile_w(30, 10, 1000, "bf16") == 256
    assert json.loads(path.read_text())["fake-gpu"]["tile_w"][autotune.tile_bucket(30, 10, 1000, "bf16")] == 128


def test_autotuner_survives_a_corrupt_cache(tmp_path):
    path = tmp_path / "tune.json"
    path.write_text("{not json")
    t = autotune.Autotuner(path=str(path), device_name="g", measure=lambda kind, **kw: kw["tile_w"])
    assert t.tile_w(10, 6, 64, "fp16") == 0
    assert json.loads(path.read_text())["g"]["tile_w"]


def test_buckets_follow_radius_channels_and_width():
    assert autotune.tile_bucket(16, 6, 100, "bf16") == "bf16/a1/C6/w0"
    assert autotune.tile_bucket(17, 6, 193, "bf16") == "bf16/a2/C6/w1"
    assert autotune.tile_bucket(48, 18, 2048, "fp16") == "fp16/a3/C18/w2"
