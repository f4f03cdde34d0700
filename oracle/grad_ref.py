"""Gradient oracle: the fast algorithm of Sec. II-III in plain PyTorch float64 on the CPU.

TEST INFRASTRUCTURE (see oracle/__init__.py).  The forward follows the same
steps as ``oracle.gcf`` (eqs. (17), (6), (7) separably with half-sample mirror,
(8), (9), (10)) and the Chebyshev fit of eqs. (16), (18), (19) with mu depending
on sigma_r, so that autograd yields the exact derivative of the approximation
with respect to the image and to sigma_r.  The paper has no gradient; this is
the definition the CUDA adjoint is checked against (itself checked against
central finite differences in the tests).
"""
import math

import numpy as np
import torch

from . import cheb_T, cheb_monomials, window_radius, mirror_index


def _mirror_indices(n, R):
    return torch.tensor([mirror_index(p, n) for p in range(-R, n + R)], dtype=torch.long)


def _taps(sigma_s, R):
    j = torch.arange(-R, R + 1, dtype=torch.float64)
    return torch.exp(-(j * j) / (2.0 * sigma_s * sigma_s))


def spatial_t(F, sigma_s, R):
    """Eq. (7), one axis at a time, on a (C, H, W) float64 tensor."""
    C, H, W = F.shape
    g = _taps(sigma_s, R).view(1, 1, -1)
    ix = _mirror_indices(W, R)
    iy = _mirror_indices(H, R)
    X = F.index_select(2, ix).reshape(C * H, 1, W + 2 * R)
    X = torch.nn.functional.conv1d(X, g).reshape(C, H, W)
    Y = X.index_select(1, iy).permute(0, 2, 1).reshape(C * W, 1, H + 2 * R)
    Y = torch.nn.functional.conv1d(Y, g).reshape(C, W, H).permute(0, 2, 1)
    return Y


def cheb_coeffs_t(N, sigma_r, L=0.0, U=255.0):
    """c_n of eq. (19) as a differentiable function of sigma_r."""
    M = N + 1
    xi = torch.tensor([math.cos(math.pi * (2 * k - 1) / (2 * M)) for k in range(1, M + 1)],
                      dtype=torch.float64)
    T = torch.tensor([[cheb_T(l, float(x)) for x in xi] for l in range(M)], dtype=torch.float64)
    a = torch.tensor(cheb_monomials(N), dtype=torch.float64)
    mu = (U - L) ** 2 / (4.0 * sigma_r * sigma_r)
    h = torch.exp(mu * xi)                               # h(mu xi_k), h = exp
    wl = torch.full((M,), 2.0 / M, dtype=torch.float64)
    wl[0] = 1.0 / M
    d = wl * (T * h.unsqueeze(0)).sum(1)                 # d_l
    n = torch.arange(M, dtype=torch.float64)
    c = (d.unsqueeze(1) * a).sum(0) * mu ** (-n)         # c_n = mu^-n sum_l d_l a_{l,n}
    return c


def gcf_t(f, sigma_s, sigma_r, N, L=0.0, U=255.0, R=None, delta=1e-12):
    """Differentiable fast approximation.  f: (H, W) float64, sigma_r: float64 scalar tensor."""
    R = window_radius(sigma_s) if R is None else R
    sigma_r = torch.as_tensor(sigma_r, dtype=torch.float64)
    tc = 0.5 * (L + U)
    c = cheb_coeffs_t(N, sigma_r, L, U)
    g = f - tc
    n = torch.arange(N + 2, dtype=torch.float64).view(-1, 1, 1)
    G = (g / sigma_r).unsqueeze(0) ** n                  # eq. (6)
    F = torch.exp(-g * g / (2.0 * sigma_r * sigma_r)).unsqueeze(0) * G
    Fb = spatial_t(F, sigma_s, R)                        # eq. (7)
    cG = c.view(-1, 1, 1) * G[: N + 1]
    P = sigma_r * (cG * Fb[1: N + 2]).sum(0)             # eq. (8)
    Q = (cG * Fb[: N + 1]).sum(0)                        # eq. (9)
    Qabs = (cG * Fb[: N + 1]).abs().sum(0)
    ok = Q.abs() >= delta * Qabs
    return torch.where(ok, P / torch.where(ok, Q, torch.ones_like(Q)) + tc, f)


def loss_and_grads(f, w, sigma_s, sigma_r, N, L=0.0, U=255.0, R=None):
    """L = sum(w * B_hat[f]); returns (L, dL/df, dL/dsigma_r) in float64."""
    ft = torch.tensor(np.asarray(f, dtype=np.float64), requires_grad=True)
    st = torch.tensor(float(sigma_r), dtype=torch.float64, requires_grad=True)
    wt = torch.tensor(np.asarray(w, dtype=np.float64))
    out = gcf_t(ft, sigma_s, st, N, L, U, R)
    loss = (wt * out).sum()
    loss.backward()
    return float(loss.detach()), ft.grad.numpy(), float(st.grad)
