"""User-facing wrappers over the C-ABI binding: a plan object, the filter call, and the
torch.autograd.Function that routes gradients through the library's adjoint."""
import warnings

import torch

from . import bfgc as B

# A range-kernel fit whose worst error reaches this (the Gaussian range kernel itself is at
# most 1) does not approximate the filter: the degree N is too low for exp on [-mu, mu],
# mu = ((U - L) / 2)^2 / sigma_r^2 (about e mu / 2 is needed)
FIT_DIVERGES = 1.0
# Beyond this mu (sigma_r below about 37 on [0, 255]) the high-degree fit needs more of the
# channels' precision than BF16's 8 significant bits keep (measured: 0.67 max-abs against the
# FP64 oracle at sigma_r = 30, N = 28; within 0.02 at sigma_r >= 40)
BF16_MU_MAX = 12.0


class GCPlan:
    """Owns a bf_gc_plan_t and its workspace tensors (allocated by PyTorch)."""

    def __init__(self, H, W, sigma_s, sigma_r, N, form="plain", precision="fp32", poly="chebyshev",
                 L=0.0, U=255.0, save_channels=False, tile_w=0, refine=True):
        self.handle = B.bf_gc_plan(H, W, sigma_s, sigma_r, N)
        try:
            B.bf_gc_plan_set(self.handle, B.BF_OPT_FORM, B.FORMS[form])
            B.bf_gc_plan_set(self.handle, B.BF_OPT_PRECISION, B.PRECISIONS[precision])
            if L != 0.0 or U != 255.0:
                B.bf_gc_plan_set(self.handle, B.BF_OPT_RANGE_U, max(U, L + 1.0))
                B.bf_gc_plan_set(self.handle, B.BF_OPT_RANGE_L, L)
                B.bf_gc_plan_set(self.handle, B.BF_OPT_RANGE_U, U)
            B.bf_gc_plan_set(self.handle, B.BF_OPT_POLY, B.POLYS[poly])
            B.bf_gc_plan_set(self.handle, B.BF_OPT_SAVE_CHANNELS, 1 if save_channels else 0)
            if tile_w:
                B.bf_gc_plan_set(self.handle, B.BF_OPT_TILE_W, int(tile_w))
            if not refine:
                B.bf_gc_plan_set(self.handle, B.BF_OPT_REFINE, 0)
        except Exception:
            B.bf_gc_plan_destroy(self.handle)
            self.handle = None
            raise
        self.H, self.W, self.sigma_s, self.sigma_r, self.N = H, W, sigma_s, sigma_r, N
        self.form, self.precision, self.poly, self.tile_w = form, precision, poly, tile_w
        self.save_channels = bool(save_channels)
        self._ws = {}
        info = self.info
        fit = info["fit_err"]
        if not fit < FIT_DIVERGES:
            warnings.warn(f"GCPlan: the degree-{N} fit of the range kernel at sigma_r={sigma_r} has worst error "
                          f"{fit:.3g}: the output does not approximate the bilateral filter; raise N",
                          RuntimeWarning, stacklevel=2)
        elif precision == "bf16" and info["mu"] > BF16_MU_MAX and info["form"] == B.BF_FORM_FUSED_TC:
            warnings.warn(f"GCPlan: BF16 channel storage at sigma_r={sigma_r} (mu = {info['mu']:.1f}) can miss the "
                          f"FP64 result by more than 0.5; precision='fp16' stays within that bound",
                          RuntimeWarning, stacklevel=2)

    def __del__(self):
        if getattr(self, "handle", None) is not None:
            B.bf_gc_plan_destroy(self.handle)
            self.handle = None

    @property
    def info(self):
        i = B.bf_gc_plan_info(self.handle)
        d = {k: getattr(i, k) for k, _ in B.bf_gc_info._fields_ if k not in ("c", "c_tilde")}
        d["c"] = [i.c[n] for n in range(i.N + 1)]
        d["c_tilde"] = [i.c_tilde[n] for n in range(i.N + 1)]
        return d

    def workspace_bytes(self):
        return B.bf_gc_workspace_size(self.handle)

    def workspace(self, kind="fwd", device=None):
        """A cached workspace tensor (uint8) large enough for the forward or the backward.

        With save_channels the forward leaves the filtered channels where the backward reads
        them, so both kinds are one buffer, sized for the larger of the two."""
        device = torch.device("cuda") if device is None else torch.device(device)
        if device.type == "cuda" and device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        fwd, bwd = self.workspace_bytes()
        if self.save_channels:
            kind, need = "shared", max(fwd, bwd)
        else:
            need = fwd if kind == "fwd" else bwd
        key = (kind, str(device))
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    def new_workspace(self, device):
        """A fresh workspace for one forward and the backward that reuses its channels."""
        fwd, bwd = self.workspace_bytes()
        return torch.empty(max(fwd, bwd, 256), dtype=torch.uint8, device=device)

    def forward(self, f, out=None, ws=None, stream=None):
        out = torch.empty_like(f) if out is None else out
        ws = self.workspace("fwd", f.device) if ws is None else ws
        return B.bf_gc_forward(self.handle, f, out, ws, stream)

    def backward(self, f, gout, gf=None, want_sigma=True, ws=None, stream=None):
        """dL/df and dL/dsigma_r.  With save_channels, `ws` must be the workspace of the last
        forward of this plan on the same f (the default is the plan's shared workspace)."""
        gf = torch.empty_like(f) if gf is None else gf
        gs = torch.zeros((), dtype=torch.float64, device=f.device) if want_sigma else None
        ws = self.workspace("bwd", f.device) if ws is None else ws
        B.bf_gc_backward(self.handle, f, gout.contiguous(), gf, gs, ws, stream)
        return gf, gs

    def diagnostics(self, ws=None, stream=None):
        ws = self.workspace("fwd") if ws is None else ws
        return B.bf_gc_diagnostics(self.handle, ws, stream)


class GCBilateral(torch.autograd.Function):
    """B_hat[f] with gradients for f and sigma_r from the library's adjoint kernels.

    `sigma_r` must equal the plan's (the plan holds the Chebyshev fit for that value); its
    gradient comes back in its own dtype and shape.  With a save_channels plan the forward
    runs in a workspace of its own, kept for the backward, which reuses its filtered channels."""

    @staticmethod
    def forward(ctx, f, sigma_r, plan):
        sr = float(sigma_r)
        if abs(sr - plan.sigma_r) > 1e-12 * abs(plan.sigma_r):
            raise ValueError(f"sigma_r = {sr} differs from the plan's {plan.sigma_r}; make a plan for it")
        f = f.contiguous()
        ws = plan.new_workspace(f.device) if plan.save_channels else None
        out = plan.forward(f, ws=ws)
        ctx.save_for_backward(f)
        ctx.plan, ctx.ws = plan, ws
        ctx.sr_meta = (sigma_r.dtype, sigma_r.shape) if isinstance(sigma_r, torch.Tensor) else None
        return out

    @staticmethod
    def backward(ctx, gout):
        (f,) = ctx.saved_tensors
        ws = ctx.ws
        if ws is None:
            ws = ctx.plan.workspace("bwd", f.device)
        gf, gs = ctx.plan.backward(f, gout, want_sigma=ctx.needs_input_grad[1], ws=ws)
        ctx.ws = None
        if gs is not None and ctx.sr_meta is not None:
            gs = gs.to(ctx.sr_meta[0]).reshape(ctx.sr_meta[1])
        return gf, gs, None


def gc_bilateral(f, sigma_s, sigma_r, N, **opts):
    """One-shot Gauss-Chebyshev bilateral filter of a float32 CUDA image (H, W)."""
    plan = GCPlan(f.shape[0], f.shape[1], sigma_s, sigma_r, N, **opts)
    return plan.forward(f.contiguous())
