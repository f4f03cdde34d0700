"""Pins of the oracle's division guard (eq. (10) with Q <= 0 or Q ~ 0; the paper assumes
Q > 0 and is silent here).  Reading: the output is the input pixel when |Q| < delta Qabs
or Qabs = 0, with Qabs = sum_n |c_n G_n Fbar_n| the sum of the absolute terms of Q of
eq. (9); otherwise P/Q + t_c.

What pins each part, independently of the formulas the oracle itself evaluates:
  * Q (value and sign) against the denominator of eq. (4) used directly in eq. (1): the
    exchange of summations of Sec. II makes sum_j g_s(j) k(tau, t_j) = exp(-tau^2/2sr^2) Q;
  * Qabs on constant images against its closed form exp(-g^2/sr^2) S^2 sum_n |c_n| x^n,
    x = (g/sr)^2 (every channel is constant there, S = the sum of the taps), i.e. the ratio
    Qabs / Q = sum_n |c_n| x^n / sum_n c_n x^n;
  * the branch itself: Qabs = 0 exactly where every channel underflows (a block far outside
    [L, U]); delta = 0 guards those pixels only; delta > 1 guards every pixel (|Q| <= Qabs by
    the triangle inequality); in between, the guarded set is {|Q| < delta Qabs}, nested in
    delta, the output there is the input pixel bit for bit and n_guard is its size.
A non-convergent fit (sigma_r = 8, N = 10: mu = 254) makes Q cancel at many pixels.
"""
import numpy as np
import pytest

import oracle
from paper_1605_02178_gb300 import synth

SS, SR, N = 1.0, 8.0, 10          # R = 3
BLOCK = (slice(4, 18), slice(30, 44))    # 14 x 14 pixels of value 1000 (u = 6.8, exp(-5947) = 0)


def guard_image():
    f = synth.rects_image(40, 48, n_rects=6, noise_std=10.0, seed=21).astype(np.float64)
    f[BLOCK] = 1000.0
    return f


def test_q_equals_the_denominator_of_the_direct_kernel():
    f = guard_image()
    _, aux = oracle.gcf(f, SS, SR, N, delta=0.0, return_pq=True)
    _, den = oracle.gcf_kernel_direct(f, SS, SR, N, return_den=True)
    e = np.exp(-(f - 127.5) ** 2 / (2 * SR ** 2))
    scale = aux["Qabs"] * e
    live = scale > 0
    assert live.mean() > 0.85                      # all but the 14 x 14 block
    assert np.all(np.abs(aux["Q"] * e - den)[live] <= 1e-10 * scale[live])
    assert np.all(den[~live] == 0.0)
    # the sign of Q changes across the image (the fit has not converged): both branches occur
    assert (aux["Q"][live] < 0).any() and (aux["Q"][live] > 0).any()


@pytest.mark.parametrize("v", [3.0, 40.0, 97.25, 127.5, 180.0, 250.0])
def test_qabs_closed_form_on_constant_images(v):
    f = np.full((9, 11), v)
    _, aux = oracle.gcf(f, SS, SR, N, delta=0.0, return_pq=True)
    c = oracle.gcf_coeffs(N, SR)
    x = ((v - 127.5) / SR) ** 2
    terms = c * x ** np.arange(N + 1)
    S = np.exp(-np.arange(-3, 4) ** 2 / (2 * SS ** 2)).sum()
    e = np.exp(-(v - 127.5) ** 2 / (2 * SR ** 2))
    want_qabs = e * S * S * np.abs(terms).sum()
    assert np.allclose(aux["Qabs"], want_qabs, rtol=1e-12, atol=0)
    if terms.sum() != 0.0:
        ratio = aux["Qabs"] / aux["Q"]
        assert np.allclose(ratio, np.abs(terms).sum() / terms.sum(), rtol=1e-9)
    if v != 127.5:                                  # the coefficients of this fit change sign
        assert (terms < 0).any() and (terms > 0).any()
        assert np.all(aux["Qabs"] > np.abs(aux["Q"]))       # mixed signs: Qabs strictly larger


def test_block_outside_the_range_is_guarded():
    """Every channel of a pixel whose whole window lies in the block underflows to 0:
    Qabs = 0, the pixel is guarded and returns its input."""
    f = guard_image()
    out, aux = oracle.gcf(f, SS, SR, N, delta=0.0, return_pq=True)
    inner = np.zeros(f.shape, bool)
    inner[7:15, 33:41] = True                      # the block minus R = 3 on each side
    assert np.all(aux["Qabs"][inner] == 0.0)
    assert np.all(aux["Qabs"][~inner] > 0.0)
    assert aux["n_guard"] == inner.sum() == 64
    assert np.all(out[inner] == 1000.0)
    ok = ~inner
    with np.errstate(invalid="ignore", divide="ignore"):
        want = aux["P"] / aux["Q"] + 127.5
    assert np.allclose(out[ok], want[ok], rtol=1e-13, atol=0)


def test_delta_above_one_guards_every_pixel():
    f = guard_image()
    out, aux = oracle.gcf(f, SS, SR, N, delta=1.0 + 1e-9, return_pq=True)
    assert np.all(np.abs(aux["Q"]) <= aux["Qabs"])
    assert aux["n_guard"] == f.size
    assert np.array_equal(out, f)


@pytest.mark.parametrize("delta", [1e-1, 1e-2, 1e-3])
def test_guarded_set_is_the_relative_threshold(delta):
    f = guard_image()
    out, aux = oracle.gcf(f, SS, SR, N, delta=delta, return_pq=True)
    Q, Qa = aux["Q"], aux["Qabs"]
    guarded = (np.abs(Q) < delta * Qa) | (Qa == 0.0)
    # the threshold splits the live pixels (the test has pixels on both sides)
    assert 64 < guarded.sum() < f.size
    assert aux["n_guard"] == guarded.sum()
    assert np.array_equal(out[guarded], f[guarded])                  # the input pixel, bit for bit
    with np.errstate(invalid="ignore", divide="ignore"):
        want = aux["P"] / Q + 127.5
    assert np.allclose(out[~guarded], want[~guarded], rtol=1e-13, atol=0)
    # not the scale of P's terms, and not t_c, decides or fills the guarded pixels
    assert not np.array_equal(guarded, (np.abs(Q) < delta * aux["Pabs"]) | (Qa == 0.0))
    assert not np.all(out[guarded] == 127.5)


def test_guarded_sets_are_nested_in_delta():
    f = guard_image()
    prev = None
    for delta in (0.0, 1e-12, 1e-6, 1e-3, 1e-1, 1.0 + 1e-9):
        out, aux = oracle.gcf(f, SS, SR, N, delta=delta, return_pq=True)
        g = out == f
        g &= (np.abs(aux["Q"]) < delta * aux["Qabs"]) | (aux["Qabs"] == 0.0)
        assert g.sum() == aux["n_guard"]
        if prev is not None:
            assert np.all(g[prev])
        prev = g
