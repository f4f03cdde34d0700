"""User-facing wrappers over the C-ABI binding: a plan object, the filter call, and the
torch.autograd.Function that routes gradients through the library's adjoint."""
import torch

from . import bfgc as B


class GCPlan:
    """Owns a bf_gc_plan_t and its workspace tensors (allocated by PyTorch)."""

    def __init__(self, H, W, sigma_s, sigma_r, N, form="plain", precision="fp32", poly="chebyshev",
                 L=0.0, U=255.0, save_channels=False, tile_w=0):
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
        except Exception:
            B.bf_gc_plan_destroy(self.handle)
            self.handle = None
            raise
        self.H, self.W, self.sigma_s, self.sigma_r, self.N = H, W, sigma_s, sigma_r, N
        self.form, self.precision, self.poly, self.tile_w = form, precision, poly, tile_w
        self._ws = {}

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
        """A cached workspace tensor (uint8) large enough for the forward or the backward."""
        device = torch.device("cuda") if device is None else torch.device(device)
        if device.type == "cuda" and device.index is None:
            device = torch.device("cuda", torch.cuda.current_device())
        need = self.workspace_bytes()[0 if kind == "fwd" else 1]
        key = (kind, str(device))
        ws = self._ws.get(key)
        if ws is None or ws.numel() < need:
            ws = torch.empty(max(need, 256), dtype=torch.uint8, device=device)
            self._ws[key] = ws
        return ws

    def forward(self, f, out=None, ws=None, stream=None):
        out = torch.empty_like(f) if out is None else out
        ws = self.workspace("fwd", f.device) if ws is None else ws
        return B.bf_gc_forward(self.handle, f, out, ws, stream)

    def backward(self, f, gout, gf=None, want_sigma=True, ws=None, stream=None):
        gf = torch.empty_like(f) if gf is None else gf
        gs = torch.zeros((), dtype=torch.float64, device=f.device) if want_sigma else None
        ws = self.workspace("bwd", f.device) if ws is None else ws
        B.bf_gc_backward(self.handle, f, gout.contiguous(), gf, gs, ws, stream)
        return gf, gs

    def diagnostics(self, ws=None, stream=None):
        ws = self.workspace("fwd") if ws is None else ws
        return B.bf_gc_diagnostics(self.handle, ws, stream)


class GCBilateral(torch.autograd.Function):
    """B_hat[f] with gradients for f and sigma_r from the library's adjoint kernels."""

    @staticmethod
    def forward(ctx, f, sigma_r, plan):
        out = plan.forward(f.contiguous())
        ctx.save_for_backward(f)
        ctx.plan = plan
        return out

    @staticmethod
    def backward(ctx, gout):
        (f,) = ctx.saved_tensors
        gf, gs = ctx.plan.backward(f.contiguous(), gout, want_sigma=ctx.needs_input_grad[1])
        return gf, (gs.to(torch.float32) if gs is not None else None), None


def gc_bilateral(f, sigma_s, sigma_r, N, **opts):
    """One-shot Gauss-Chebyshev bilateral filter of a float32 CUDA image (H, W)."""
    plan = GCPlan(f.shape[0], f.shape[1], sigma_s, sigma_r, N, **opts)
    return plan.forward(f.contiguous())
