"""Row strips of one image over several ranks, with a halo exchange of image rows.

Every step of the filter is per pixel except the spatial Gaussian of eq. (7), which reaches
R = ceil(3 sigma_s) rows up and down.  So rank k can own rows [y0, y1) of the output if it
has the input rows [y0 - R, y1 + R) (clamped to the image): the rows within R of its strip
come from the ranks that own them, and the forward runs on the extended strip as if it were
an image of its own.  Its half-sample mirror extension (Sec. I) is then right at the image's
true top and bottom, and wrong only at a cut inside the image; the rows that the wrong
extension reaches are the halo rows, which the rank drops.  For the exact forms (plain,
fused, tensor-core) the owned rows are what the whole image gives; the recursive stand-in
reaches beyond R rows, so it is refused here.

The adjoint reaches twice as far: dL/df at an owned row sums the contributions of the
outputs within R of it, and each of those needs the input within R of itself.  A rank takes
f with a 2R halo and the upstream gradient w with an R halo (zero beyond), and keeps its own
rows of dL/df.  dL/dsigma_r is a sum over pixels: each rank sums its own rows (w zero
elsewhere, f with an R halo) and the ranks add their sums (all-reduce).

The exchange is the one collective: each rank sends every other rank the rows of its strip
that the other's extended range covers (usually R rows to each neighbour; more ranks when
a strip is thinner than the halo), with point-to-point sends and receives of torch.distributed
(NCCL for device tensors, gloo for host tensors).
"""
import math

import torch
import torch.distributed as dist

from . import api, bfgc as B


def window_radius(sigma_s):
    """R = ceil(3 sigma_s), as the plan computes it (a 1e-9 slack absorbs representation error)."""
    return int(math.ceil(3.0 * sigma_s - 1e-9))


def strip_rows(H, world, rank):
    """Rows [y0, y1) of rank `rank` when H rows are split as evenly as possible over `world`."""
    base, extra = divmod(H, world)
    y0 = rank * base + min(rank, extra)
    return y0, y0 + base + (1 if rank < extra else 0)


def halo_range(H, y0, y1, halo):
    """The strip [y0, y1) extended by `halo` rows on each side, clamped to [0, H)."""
    return max(0, y0 - halo), min(H, y1 + halo)


def exchange_rows(x_own, H, halo, group=None):
    """Rows [e0, e1) = halo_range(strip of this rank, halo) of a row-distributed (H, W) array of
    which this rank holds its own strip `x_own`; the other rows are received from their owners."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    y0, y1 = strip_rows(H, world, rank)
    if x_own.shape[0] != y1 - y0:
        raise ValueError(f"rank {rank} holds {x_own.shape[0]} rows, its strip has {y1 - y0}")
    x_own = x_own.contiguous()
    e0, e1 = halo_range(H, y0, y1, halo)
    x_ext = x_own.new_empty((e1 - e0,) + tuple(x_own.shape[1:]))
    x_ext[y0 - e0:y1 - e0] = x_own
    sends, recvs = [], []
    for peer in range(world):
        if peer == rank:
            continue
        p0, p1 = strip_rows(H, world, peer)
        q0, q1 = halo_range(H, p0, p1, halo)
        s0, s1 = max(q0, y0), min(q1, y1)           # my rows the peer needs
        if s0 < s1:
            rows = x_own[s0 - y0:s1 - y0].contiguous()   # held until its send completes
            sends.append((dist.isend(rows, dst=_global(peer, group), group=group), rows))
        r0, r1 = max(e0, p0), min(e1, p1)           # the peer's rows I need
        if r0 < r1:
            buf = x_own.new_empty((r1 - r0,) + tuple(x_own.shape[1:]))
            recvs.append((dist.irecv(buf, src=_global(peer, group), group=group), buf, r0 - e0))
    for req, buf, at in recvs:
        req.wait()
        x_ext[at:at + buf.shape[0]] = buf
    for req, _ in sends:
        req.wait()
    return x_ext


def _global(peer, group):
    return peer if group is None else dist.get_global_rank(group, peer)


def _aligned(x):
    """x as a contiguous tensor whose data starts on a 16-byte boundary (what the C ABI asks
    for); a row slice of an image whose width is not a multiple of 4 is copied."""
    x = x.contiguous()
    return x if x.data_ptr() % 16 == 0 else x.clone()


def _check_exact(plan):
    if plan.info["form"] == B.BF_FORM_RECURSIVE:
        raise ValueError("the recursive form reaches beyond R rows: row strips need an exact form")


def forward_strip(f_ext, ext_range, own_range, sigma_s, sigma_r, N, filter_fn=None, **plan_opts):
    """Rows own_range = [y0, y1) of the filtered image from its rows ext_range = [e0, e1)
    (= halo_range(H, y0, y1, R)).  filter_fn(f_ext) replaces the library forward."""
    (e0, e1), (y0, y1) = ext_range, own_range
    if y1 <= y0:                                    # more ranks than rows: an empty strip
        return f_ext[:0]
    if filter_fn is None:
        plan = api.GCPlan(e1 - e0, f_ext.shape[1], sigma_s, sigma_r, N, **plan_opts)
        _check_exact(plan)
        out = plan.forward(_aligned(f_ext))
    else:
        out = filter_fn(f_ext)
    return out[y0 - e0:y1 - e0]


def forward_strips(f_own, H, sigma_s, sigma_r, N, group=None, filter_fn=None, **plan_opts):
    """The filtered rows of this rank's strip of an H-row image (see the module text)."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    R = window_radius(sigma_s)
    y0, y1 = strip_rows(H, world, rank)
    f_ext = exchange_rows(f_own, H, R, group)
    return forward_strip(f_ext, halo_range(H, y0, y1, R), (y0, y1), sigma_s, sigma_r, N, filter_fn, **plan_opts)


def backward_strip(f_ext2, w_ext1, H, own_range, sigma_s, sigma_r, N, grad_fn=None, **plan_opts):
    """(dL/df on own_range, this strip's part of dL/dsigma_r) for L = sum(w * filter(f)), from f
    on halo_range(H, y0, y1, 2R) and w on halo_range(H, y0, y1, R).  grad_fn(f, w) -> (dL/df,
    dL/dsigma_r) replaces the library adjoint."""
    y0, y1 = own_range
    if y1 <= y0:
        return f_ext2[:0], 0.0
    R = window_radius(sigma_s)
    e0, e1 = halo_range(H, y0, y1, 2 * R)
    a0, a1 = halo_range(H, y0, y1, R)
    if grad_fn is None:
        def grad_fn(f, w):
            plan = api.GCPlan(f.shape[0], f.shape[1], sigma_s, sigma_r, N, **plan_opts)
            _check_exact(plan)
            return plan.backward(_aligned(f), _aligned(w))
    # dL/df: f with the 2R halo, w with the R halo and zero beyond
    w2 = torch.zeros_like(f_ext2)
    w2[a0 - e0:a1 - e0] = w_ext1
    gf = grad_fn(f_ext2, w2)[0][y0 - e0:y1 - e0]
    # dL/dsigma_r over the owned rows: f with the R halo, w zero outside the strip
    w1 = torch.zeros_like(w_ext1)
    w1[y0 - a0:y1 - a0] = w_ext1[y0 - a0:y1 - a0]
    gs = grad_fn(f_ext2[a0 - e0:a1 - e0], w1)[1]
    return gf, gs


def backward_strips(f_own, w_own, H, sigma_s, sigma_r, N, group=None, grad_fn=None, **plan_opts):
    """(dL/df on this rank's strip, dL/dsigma_r of the whole image) for L = sum(w * filter(f)),
    with f and w row-distributed as strip_rows gives."""
    world, rank = dist.get_world_size(group), dist.get_rank(group)
    R = window_radius(sigma_s)
    y0, y1 = strip_rows(H, world, rank)
    f2 = exchange_rows(f_own, H, 2 * R, group)
    w1 = exchange_rows(w_own, H, R, group)
    gf, gs = backward_strip(f2, w1, H, (y0, y1), sigma_s, sigma_r, N, grad_fn, **plan_opts)
    total = torch.as_tensor(gs, dtype=torch.float64, device=f_own.device).reshape(1).clone()
    dist.all_reduce(total, group=group)
    return gf, total[0]
