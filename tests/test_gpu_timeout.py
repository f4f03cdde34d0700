"""The bounded waits of the pipelined tensor-core kernels, made to run out on purpose.

BF_OPT_STALL makes one role withhold its first signal while nothing asynchronous is
outstanding for it (1: the row pass's first build group never hands over its first tile, so
the MMA issuer waits on it; 2: the column pass's TMA producer never loads its first stage).
With BF_OPT_WAIT_US = 2000 the waiting role gives up after 2 ms, raises the kernel's abort
flag, every role returns, and bf_gc_diagnostics reports BF_ERR_TIMEOUT with that kernel's
error bit (4: row pass with the Toeplitz operand in tensor memory, 8: column pass with channel
pairs).  The context stays usable: a normal forward afterwards matches the FP64 oracle.
"""
import numpy as np
import pytest
import torch

import oracle
from paper_1605_02178_gb300 import api, bfgc, synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("stall,bit", [(1, 4), (2, 8)])
def test_a_withheld_signal_ends_in_a_timeout_not_a_hang(stall, bit):
    H, W, ss, sr, N = 300, 420, 3.0, 50.0, 12
    f = synth.rects_image(H, W, n_rects=8, noise_std=10.0, seed=11)
    ft = torch.from_numpy(f).cuda()
    plan = api.GCPlan(H, W, ss, sr, N, form="fused_tc", precision="fp16", refine=False)
    bfgc.bf_gc_plan_set(plan.handle, bfgc.BF_OPT_WAIT_US, 2000.0)
    bfgc.bf_gc_plan_set(plan.handle, bfgc.BF_OPT_STALL, stall)
    ws = plan.workspace("fwd")
    plan.forward(ft, ws=ws)
    d = bfgc.bf_gc_diag()
    st = bfgc.lib().bf_gc_diagnostics(plan.handle, bfgc._ptr(ws), bfgc.ctypes.byref(d), bfgc._stream(None))
    assert st == bfgc.BF_ERR_TIMEOUT
    assert d.error_flags & bit
    torch.cuda.synchronize()
    # the context is intact: the same workload on a normal plan matches the oracle
    ref = oracle.gcf(f, ss, sr, N)
    good = api.GCPlan(H, W, ss, sr, N, form="fused_tc", precision="fp16")
    out = good.forward(ft)
    torch.cuda.synchronize()
    assert np.abs(out.cpu().numpy().astype(np.float64) - ref).max() <= 0.05
    dg = good.diagnostics()
    assert dg["error_flags"] == 0
