"""Batches of independent images, each with its own size, sigma_s, sigma_r and N, filtered
as one CUDA graph through bf_gc_batch_* (include/bfgc.h).

The paper filters one image at a time (Sec. III); a batch runs the same per-image method.
mode="branches": per-image forwards on concurrent graph branches, so every image's result
equals that of a single bf_gc_forward with the same plan, bit for bit; branch counts and
row-pass tile widths come from the Autotuner (autotune.py) when one is given.
mode="persistent" (tensor-core form): one launch of each pass over a device work list of
(image, tile) items; each image equals its own forward up to the FP32 summation order of the
banded products, with the FP32 guard of eq. (10) in place of the FP64 refinement.
"""
import torch

from . import bfgc as B
from .api import GCPlan

DEFAULT_BRANCHES = 8


class GCBatch:
    """Owns one GCPlan per image, the bf_gc_batch_t over them and the batch workspace.

    specs: sequence of dicts with H, W, sigma_s, sigma_r, N and optionally tile_w (row-pass
    tile width of the tensor-core form; 0 = default).  form, precision, poly and refine (the
    plans' FP64 refinement, branches mode) apply to every image.
    """

    def __init__(self, specs, form="fused_tc", precision="bf16", poly="chebyshev", branches=None,
                 tuner=None, device=None, mode="branches", refine=True):
        if not specs:
            raise ValueError("empty batch")
        if mode not in ("branches", "persistent"):
            raise ValueError(f"mode {mode!r}: 'branches' or 'persistent'")
        self.form, self.precision, self.poly, self.mode = form, precision, poly, mode
        self.device = torch.device("cuda", torch.cuda.current_device()) if device is None else torch.device(device)
        self.tuner = tuner
        self.plans = []
        for s in specs:
            tw = int(s.get("tile_w", 0))
            plan = GCPlan(s["H"], s["W"], s["sigma_s"], s["sigma_r"], s["N"], form=form, precision=precision,
                          poly=poly, refine=refine)
            if tw == 0 and tuner is not None and form == "fused_tc" and mode == "branches":
                info = plan.info
                tw = tuner.tile_w(info["R"], info["C"], s["W"], precision)
            if tw:
                B.bf_gc_plan_set(plan.handle, B.BF_OPT_TILE_W, tw)
                plan.tile_w = tw
            self.plans.append(plan)
        self.handle = None
        self.ws = None
        self._make(DEFAULT_BRANCHES if branches is None else int(branches))
        self._tuned = branches is not None or tuner is None or mode == "persistent"

    def _make(self, branches):
        if self.handle is not None:
            B.bf_gc_batch_destroy(self.handle)
            self.handle = None
        if self.mode == "persistent":
            self.handle = B.bf_gc_batch_create_persistent([p.handle for p in self.plans])
        else:
            self.handle = B.bf_gc_batch_create([p.handle for p in self.plans], branches)
        self.branches = branches
        need = max(B.bf_gc_batch_workspace_size(self.handle), 256)
        if self.ws is None or self.ws.numel() < need:
            self.ws = None
            self.ws = torch.empty(need, dtype=torch.uint8, device=self.device)

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            B.bf_gc_batch_destroy(self.handle)
            self.handle = None

    def __len__(self):
        return len(self.plans)

    @property
    def pixels(self):
        return sum(p.H * p.W for p in self.plans)

    def diagnostics(self, stream=None):
        """Counters of the last forward (persistent mode: all images together)."""
        return self.plans[0].diagnostics(self.ws, stream)

    def info(self):
        """(branch of each image, CUDA graphs captured so far)."""
        return B.bf_gc_batch_info(self.handle, len(self.plans))

    def forward(self, fs, outs=None, stream=None):
        """outs[i] = B_hat[fs[i]] for every image (fs: float32 CUDA tensors (H_i, W_i)).

        The first call with a given set of tensors captures the graph (and, with a tuner and no
        fixed branch count, first times the candidate branch counts on these tensors)."""
        if len(fs) != len(self.plans):
            raise ValueError(f"batch of {len(self.plans)} images, got {len(fs)} inputs")
        for f, p in zip(fs, self.plans):
            if tuple(f.shape) != (p.H, p.W):
                raise ValueError(f"image of shape {tuple(f.shape)} where ({p.H}, {p.W}) was planned")
        outs = [torch.empty_like(f) for f in fs] if outs is None else outs
        if not self._tuned:
            self._tuned = True
            best = self.tuner.branches(self.signature(), lambda k: self._time_branches(k, fs, outs, stream))
            if best != self.branches:
                self._make(best)
        B.bf_gc_batch_forward(self.handle, fs, outs, self.ws, stream)
        return outs

    def signature(self):
        """Cache key of the batch's composition (count, pixels, parameters), for the tuner."""
        px = self.pixels
        return f"{self.form}/{self.precision}/n{len(self.plans)}/mpx{round(px / 1e6)}/" \
               f"h{hash(tuple((p.H, p.W, p.sigma_s, p.sigma_r, p.N) for p in self.plans)) & 0xffffffff:08x}"

    def _time_branches(self, k, fs, outs, stream, reps=3):
        self._make(k)
        s = torch.cuda.current_stream() if stream is None else stream
        B.bf_gc_batch_forward(self.handle, fs, outs, self.ws, s)       # capture + warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(reps):
            B.bf_gc_batch_forward(self.handle, fs, outs, self.ws, s)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / reps
