"""FP64 CPU oracle of the Gauss-Chebyshev bilateral filter (Ghosh & Chaudhury 2016).

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this package.  The product library never calls it
and shares no code with it.

The arithmetic lives in ``bfgc_oracle.c`` (plain C, double precision); this
module only marshals numpy arrays to it.  ``grad_ref`` holds the gradient
oracle (plain PyTorch CPU float64 autograd over the same algorithm).

Paper sections followed (see the C file for the per-function citations):
  eq. (1)            exact bilateral filter           -> exact_bf, exact_bf_at
  eqs. (11)-(19)     Chebyshev fit on [-mu, mu]       -> cheb_fit
  eqs. (6)-(10),(17) fast algorithm (GCF)             -> gcf, gcf_at
  eq. (4) + (19)     approximate kernel, direct       -> gcf_kernel_direct
  eq. (7)            spatial Gaussian                 -> spatial
"""
import ctypes
import math
import os

import numpy as np

from . import build as _build

_LIB = None
_dp = ctypes.POINTER(ctypes.c_double)
_i64p = ctypes.POINTER(ctypes.c_int64)

SPATIAL_MODES = {"separable": 0, "recursive": 1, "2d": 2}


def _lib():
    global _LIB
    if _LIB is None:
        path = _build.build()
        lib = ctypes.CDLL(path)
        I, D, L = ctypes.c_int, ctypes.c_double, ctypes.c_long
        lib.oracle_exact_bf.argtypes = [_dp, I, I, D, D, I, _dp]
        lib.oracle_exact_bf_at.argtypes = [_dp, I, I, D, D, I, _i64p, L, _dp]
        lib.oracle_cheb_T.argtypes = [I, D]
        lib.oracle_cheb_T.restype = D
        lib.oracle_cheb_monomials.argtypes = [I, _dp]
        lib.oracle_cheb_fit.argtypes = [I, D, _dp, _dp, _dp, _dp]
        lib.oracle_spatial_2d.argtypes = [_dp, I, I, D, I, _dp]
        lib.oracle_spatial_separable.argtypes = [_dp, I, I, D, I, _dp]
        lib.oracle_spatial_recursive.argtypes = [_dp, I, I, D, I, _dp]
        lib.oracle_yvv_coeffs.argtypes = [D, _dp]
        lib.oracle_yvv_1d.argtypes = [_dp, L, D, L, _dp]
        lib.oracle_gcf.argtypes = [_dp, I, I, D, D, I, I, D, D, _dp, D, I, _dp, _dp, _dp, _dp, _dp,
                                   ctypes.POINTER(ctypes.c_long)]
        lib.oracle_gcf_at.argtypes = [_dp, I, I, D, D, I, I, D, D, _dp, D, _i64p, L, _dp, _dp, _dp]
        lib.oracle_gcf_kernel_direct.argtypes = [_dp, I, I, D, D, I, I, D, D, _dp, _dp, _dp]
        lib.oracle_mirror_index.argtypes = [L, L]
        _LIB = lib
    return _LIB


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _check(rc, what):
    if rc != 0:
        raise RuntimeError(f"oracle {what} failed with code {rc}")


def window_radius(sigma_s: float) -> int:
    """Half-width of the spatial window, W = 3 sigma_s of Sec. I, rounded up."""
    return int(math.ceil(3.0 * sigma_s - 1e-9))


def num_threads() -> int:
    return _lib().oracle_num_threads()


def mirror_index(p: int, n: int) -> int:
    return _lib().oracle_mirror_index(p, n)


# ----------------------------------------------------------------------------- eq. (1)
def exact_bf(f, sigma_s, sigma_r, R=None):
    f = _f64(f)
    H, W = f.shape
    R = window_radius(sigma_s) if R is None else R
    out = np.empty_like(f)
    _check(_lib().oracle_exact_bf(_ptr(f), H, W, sigma_s, sigma_r, R, _ptr(out)), "exact_bf")
    return out


def exact_bf_at(f, idx, sigma_s, sigma_r, R=None):
    f = _f64(f)
    H, W = f.shape
    R = window_radius(sigma_s) if R is None else R
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out = np.empty(idx.shape[0], dtype=np.float64)
    _check(_lib().oracle_exact_bf_at(_ptr(f), H, W, sigma_s, sigma_r, R,
                                     idx.ctypes.data_as(_i64p), idx.shape[0], _ptr(out)),
           "exact_bf_at")
    return out


# ----------------------------------------------------------------------------- eqs. (11)-(19)
def cheb_T(l, x):
    return _lib().oracle_cheb_T(int(l), float(x))


def cheb_monomials(N):
    a = np.empty((N + 1, N + 1))
    _check(_lib().oracle_cheb_monomials(N, _ptr(a)), "cheb_monomials")
    return a


def cheb_fit(N, mu):
    """Nodes xi_k, coefficients d_l, monomial table a_{l,n}, and c_n of eq. (19)."""
    xi, d, c = np.empty(N + 1), np.empty(N + 1), np.empty(N + 1)
    a = np.empty((N + 1, N + 1))
    _check(_lib().oracle_cheb_fit(N, float(mu), _ptr(xi), _ptr(d), _ptr(a), _ptr(c)), "cheb_fit")
    return {"xi": xi, "d": d, "a": a, "c": c}


def interval_mu(sigma_r, L=0.0, U=255.0):
    """mu = (U - L)^2 / (4 sigma_r^2), Sec. III-B."""
    return (U - L) ** 2 / (4.0 * sigma_r ** 2)


def gcf_coeffs(N, sigma_r, L=0.0, U=255.0):
    return cheb_fit(N, interval_mu(sigma_r, L, U))["c"]


def taylor_coeffs(N):
    """c_n = 1/n!, the Gauss-polynomial (Taylor) choice recalled in Sec. II."""
    return np.array([1.0 / math.factorial(n) for n in range(N + 1)])


# ----------------------------------------------------------------------------- eq. (7)
def spatial(F, sigma_s, R=None, mode="separable"):
    F = _f64(F)
    H, W = F.shape
    R = window_radius(sigma_s) if R is None else R
    out = np.empty_like(F)
    fn = {"separable": _lib().oracle_spatial_separable, "2d": _lib().oracle_spatial_2d,
          "recursive": _lib().oracle_spatial_recursive}[mode]
    _check(fn(_ptr(F), H, W, float(sigma_s), R, _ptr(out)), "spatial")
    return out


def yvv_coeffs(sigma):
    b = np.empty(5)
    _check(_lib().oracle_yvv_coeffs(float(sigma), _ptr(b)), "yvv_coeffs")
    return b


def yvv_1d(x, sigma, P):
    x = _f64(x)
    out = np.empty_like(x)
    _check(_lib().oracle_yvv_1d(_ptr(x), x.shape[0], float(sigma), int(P), _ptr(out)), "yvv_1d")
    return out


# ----------------------------------------------------------------------------- eqs. (6)-(10)
def gcf(f, sigma_s, sigma_r, N, L=0.0, U=255.0, c=None, delta=1e-12, spatial="separable",
        R=None, return_pq=False):
    """Fast approximation of eq. (1): eqs. (17), (6), (7), (8), (9), (10), un-centring.

    ``c`` defaults to the Gauss-Chebyshev coefficients of eq. (19).
    """
    f = _f64(f)
    H, W = f.shape
    R = window_radius(sigma_s) if R is None else R
    c = gcf_coeffs(N, sigma_r, L, U) if c is None else _f64(c)
    out = np.empty_like(f)
    P, Q, Qa, Pa = (np.empty_like(f) for _ in range(4)) if return_pq else (None,) * 4
    ng = ctypes.c_long(0)
    _check(_lib().oracle_gcf(_ptr(f), H, W, float(sigma_s), float(sigma_r), int(N), R, float(L),
                             float(U), _ptr(c), float(delta), SPATIAL_MODES[spatial], _ptr(out),
                             _ptr(P) if P is not None else None,
                             _ptr(Q) if Q is not None else None,
                             _ptr(Qa) if Qa is not None else None,
                             _ptr(Pa) if Pa is not None else None, ctypes.byref(ng)), "gcf")
    if return_pq:
        return out, {"P": P, "Q": Q, "Qabs": Qa, "Pabs": Pa, "n_guard": ng.value}
    return out


def gcf_at(f, idx, sigma_s, sigma_r, N, L=0.0, U=255.0, c=None, delta=1e-12, R=None,
           return_pq=False):
    f = _f64(f)
    H, W = f.shape
    R = window_radius(sigma_s) if R is None else R
    c = gcf_coeffs(N, sigma_r, L, U) if c is None else _f64(c)
    idx = np.ascontiguousarray(idx, dtype=np.int64)
    out, P, Q = (np.empty(idx.shape[0]) for _ in range(3))
    _check(_lib().oracle_gcf_at(_ptr(f), H, W, float(sigma_s), float(sigma_r), int(N), R,
                                float(L), float(U), _ptr(c), float(delta),
                                idx.ctypes.data_as(_i64p), idx.shape[0], _ptr(out), _ptr(P),
                                _ptr(Q)), "gcf_at")
    if return_pq:
        return out, {"P": P, "Q": Q}
    return out


def gcf_kernel_direct(f, sigma_s, sigma_r, N, L=0.0, U=255.0, c=None, R=None, return_den=False):
    """Eq. (4) with the coefficients of eq. (19) used as the range kernel of eq. (1).  With
    return_den, also the denominator sum_j g_s(j) k(g(i), g(i - j)) per pixel."""
    f = _f64(f)
    H, W = f.shape
    R = window_radius(sigma_s) if R is None else R
    c = gcf_coeffs(N, sigma_r, L, U) if c is None else _f64(c)
    out = np.empty_like(f)
    den = np.empty_like(f) if return_den else None
    _check(_lib().oracle_gcf_kernel_direct(_ptr(f), H, W, float(sigma_s), float(sigma_r), int(N),
                                           R, float(L), float(U), _ptr(c), _ptr(out),
                                           _ptr(den) if den is not None else None),
           "gcf_kernel_direct")
    return (out, den) if return_den else out


# ----------------------------------------------------------------------------- Sec. IV metric
def mse_db(a, b):
    """10 log10 of the mean squared difference (Sec. IV)."""
    d = np.asarray(a, dtype=np.float64) - np.asarray(b, dtype=np.float64)
    m = float(np.mean(d * d))
    return -math.inf if m == 0.0 else 10.0 * math.log10(m)


def psnr_db(a, b, peak=255.0):
    return 20.0 * math.log10(peak) - mse_db(a, b)
