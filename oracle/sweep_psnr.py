"""Accuracy of the Gauss-Chebyshev approximation over the 4K sweep, from the FP64 oracle alone.

TEST INFRASTRUCTURE (see oracle/__init__.py): a study run by hand on the host, never by
the library.  For each of sigma_s in {5, 10, 20} x sigma_r in {10, 30, 50} x N in {5, 10, 20},
and the anchor sigma_s = 10, sigma_r = 30, N = 28, on the 4K edge + smooth workload
(3840x2160), it evaluates the fast algorithm of eqs. (6)-(10) (``gcf_at``, eq. (7) as the
literal double sum) and the exact filter of eq. (1) (``exact_bf_at``) at the same sampled
pixels, 16 evenly spaced rows (the first and last included) times every 4th column, and
prints one JSON line per configuration with the PSNR of the approximation against the
exact filter over those pixels and the largest absolute difference.

These are properties of the approximation itself (FP64): the FP32 GPU forms are held to
1e-3 of the same oracle, so their PSNR against the exact filter is this one wherever this
is below about 100 dB.

    python -m oracle.sweep_psnr > sweep_psnr.jsonl
"""
import json
import math
import sys
import time

import numpy as np

from . import exact_bf_at, gcf_at, window_radius


def sample_indices(H, W, rows=16, col_step=4):
    ys = np.linspace(0, H - 1, rows).round().astype(np.int64)
    xs = np.arange(0, W, col_step, dtype=np.int64)
    return (ys[:, None] * W + xs[None, :]).reshape(-1)


def configs():
    out = [(ss, sr, N) for ss in (5.0, 10.0, 20.0) for sr in (10.0, 30.0, 50.0) for N in (5, 10, 20)]
    out.append((10.0, 30.0, 28))
    return out


def main():
    sys.path.insert(0, ".")
    from paper_1605_02178_gb300 import synth      # seeded generator only: no filter arithmetic
    f = synth.workload("uhd")["f"]
    H, W = f.shape
    idx = sample_indices(H, W)
    exact = {}
    for ss, sr, N in configs():
        t0 = time.perf_counter()
        if (ss, sr) not in exact:
            exact[(ss, sr)] = exact_bf_at(f, idx, ss, sr)
        ex = exact[(ss, sr)]
        ap = gcf_at(f, idx, ss, sr, N)
        mse = float(np.mean((ap - ex) ** 2))
        print(json.dumps({
            "study": "sweep_accuracy", "image": "uhd 3840x2160", "sigma_s": ss, "R": window_radius(ss),
            "sigma_r": sr, "N": N, "pixels": int(idx.size),
            "psnr_vs_exact_db": float("inf") if mse == 0.0 else 10.0 * math.log10(255.0 ** 2 / mse),
            "maxabs_vs_exact": float(np.abs(ap - ex).max()),
            "seconds": time.perf_counter() - t0}), flush=True)


if __name__ == "__main__":
    main()
