"""Row strips of one image over ranks (paper_1605_02178_gb300/strips.py) on CPU: the split and
halo bookkeeping, and, as gloo process groups of 2 and 3 ranks, the halo exchange with the
FP64 oracle standing in for the per-strip filter and its gradient.  The strips put together
must give what the oracle gives on the whole image: the forward, dL/df and dL/dsigma_r
(L = sum(w * filter(f))), including strips thinner than the halo, whose rows come from
several ranks."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1605_02178_gb300 import strips

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.mark.parametrize("H,world", [(1, 1), (10, 3), (29, 3), (7, 7), (5, 8), (2160, 8)])
def test_strips_cover_the_image_once_and_are_balanced(H, world):
    rows = [strips.strip_rows(H, world, k) for k in range(world)]
    assert rows[0][0] == 0 and rows[-1][1] == H
    for (a0, a1), (b0, b1) in zip(rows, rows[1:]):
        assert a1 == b0
    sizes = [b - a for a, b in rows]
    assert max(sizes) - min(sizes) <= 1


def test_halo_range_clamps_at_the_image():
    assert strips.halo_range(100, 0, 30, 6) == (0, 36)
    assert strips.halo_range(100, 30, 60, 6) == (24, 66)
    assert strips.halo_range(100, 90, 100, 12) == (78, 100)
    assert strips.halo_range(10, 4, 7, 30) == (0, 10)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


CASES = [  # H, W, sigma_s, sigma_r, N
    (29, 17, 2.0, 40.0, 8),     # R = 6, strips of 9-15 rows
    (10, 13, 2.0, 50.0, 6),     # strips of 3-5 rows, thinner than the halo (6, and 12 for the adjoint)
    (2, 9, 1.0, 50.0, 4),       # fewer rows than three ranks: one strip is empty
]


def _worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import grad_ref
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    res = []
    for H, W, ss, sr, N in CASES:
        f = np.random.default_rng(H * 100 + W).uniform(0, 255, (H, W))
        w = np.random.default_rng(H * 100 + W + 1).standard_normal((H, W))
        y0, y1 = strips.strip_rows(H, world, rank)

        def filt(fe):
            return torch.from_numpy(oracle.gcf(fe.numpy(), ss, sr, N))

        def grad(fe, we):
            _, gf, gs = grad_ref.loss_and_grads(fe.numpy(), we.numpy(), ss, sr, N)
            return torch.from_numpy(gf), gs
        out = strips.forward_strips(torch.from_numpy(f[y0:y1].copy()), H, ss, sr, N, filter_fn=filt)
        gf, gs = strips.backward_strips(torch.from_numpy(f[y0:y1].copy()), torch.from_numpy(w[y0:y1].copy()),
                                        H, ss, sr, N, grad_fn=grad)
        res.append((out.numpy(), gf.numpy(), float(gs)))
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, res))


@pytest.mark.parametrize("world", [2, 3])
def test_strips_over_gloo_ranks_equal_the_whole_image(world):
    sys.path.insert(0, ROOT)
    import oracle
    from oracle import grad_ref
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for i, (H, W, ss, sr, N) in enumerate(CASES):
        f = np.random.default_rng(H * 100 + W).uniform(0, 255, (H, W))
        w = np.random.default_rng(H * 100 + W + 1).standard_normal((H, W))
        ref = oracle.gcf(f, ss, sr, N)
        _, gf_ref, gs_ref = grad_ref.loss_and_grads(f, w, ss, sr, N)
        out = np.concatenate([got[k][i][0] for k in range(world)])
        gf = np.concatenate([got[k][i][1] for k in range(world)])
        assert out.shape == (H, W) and gf.shape == (H, W)
        assert np.abs(out - ref).max() <= 1e-9
        assert np.abs(gf - gf_ref).max() <= 1e-9 * max(1.0, np.abs(gf_ref).max())
        for k in range(world):                       # every rank holds the all-reduced sum
            assert abs(got[k][i][2] - gs_ref) <= 1e-9 * max(1.0, abs(gs_ref))


def _group_worker(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    members = [1, 2, 3]
    group = dist.new_group(members)
    res = None
    if rank in members:
        H, W, ss, sr, N = CASES[0]
        f = np.random.default_rng(H * 100 + W).uniform(0, 255, (H, W))
        k = dist.get_rank(group)
        y0, y1 = strips.strip_rows(H, len(members), k)
        out = strips.forward_strips(torch.from_numpy(f[y0:y1].copy()), H, ss, sr, N, group=group,
                                    filter_fn=lambda fe: torch.from_numpy(oracle.gcf(fe.numpy(), ss, sr, N)))
        res = (k, out.numpy())
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, res))


def test_strips_over_a_subgroup_of_ranks():
    """Strips over a process subgroup (global ranks 1-3 of 4): peers are addressed by their
    global ranks, strips by their ranks in the group."""
    sys.path.insert(0, ROOT)
    import oracle
    world, port = 4, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_group_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=300) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got[0] is None
    parts = sorted(v for v in got.values() if v is not None)
    H, W, ss, sr, N = CASES[0]
    f = np.random.default_rng(H * 100 + W).uniform(0, 255, (H, W))
    out = np.concatenate([p[1] for p in parts])
    assert np.abs(out - oracle.gcf(f, ss, sr, N)).max() <= 1e-9
