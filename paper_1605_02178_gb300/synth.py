"""Seeded synthetic grayscale images (numpy only, no filter arithmetic).

These stand in for the test images the paper uses (Checker, Testpat, Barbara
in Sec. IV), which are not available: piecewise-constant fields with sharp
edges, smooth 1/f fields, and noise, in the intensity range [0, 255].

The same generators feed both the CUDA path and the FP64 oracle in tests and
in the benchmark; nothing here computes any part of the filter.
"""
import numpy as np

__all__ = ["rects_image", "edge_smooth_image", "weight_map", "checkerboard",
           "batch_specs", "workload"]


def rects_image(H, W, n_rects=20, noise_std=10.0, seed=0):
    """Background level, then axis-aligned rectangles of random level, then noise.

    Rectangles: top-left uniform on the frame, height and width uniform in
    {16..256}, level uniform in [0, 255], clipped to the frame, painted in order.
    """
    rng = np.random.default_rng(seed)
    img = np.full((H, W), rng.uniform(0.0, 255.0), dtype=np.float64)
    for _ in range(n_rects):
        y0 = int(rng.integers(0, H))
        x0 = int(rng.integers(0, W))
        h = int(rng.integers(16, 257))
        w = int(rng.integers(16, 257))
        img[y0:min(H, y0 + h), x0:min(W, x0 + w)] = rng.uniform(0.0, 255.0)
    img += rng.normal(0.0, noise_std, size=(H, W))
    return np.ascontiguousarray(np.clip(img, 0.0, 255.0), dtype=np.float32)


def _edge_field(H, W, rng):
    def cuts(n):
        edges = [0]
        while edges[-1] < n:
            edges.append(edges[-1] + int(rng.integers(8, 65)))
        return np.minimum(np.array(edges), n)
    ys, xs = cuts(H), cuts(W)
    levels = rng.uniform(0.0, 255.0, size=(len(ys) - 1, len(xs) - 1))
    row_cell = np.searchsorted(ys, np.arange(H), side="right") - 1
    col_cell = np.searchsorted(xs, np.arange(W), side="right") - 1
    return levels[row_cell][:, col_cell]


def _smooth_field(H, W, rng):
    noise = rng.normal(size=(H, W))
    spec = np.fft.rfft2(noise)
    ky = np.fft.fftfreq(H)[:, None]
    kx = np.fft.rfftfreq(W)[None, :]
    k = np.sqrt(ky * ky + kx * kx)
    k[0, 0] = 1.0
    spec = spec / k
    spec[0, 0] = 0.0
    field = np.fft.irfft2(spec, s=(H, W))
    lo, hi = field.min(), field.max()
    return (field - lo) / (hi - lo) * 255.0 if hi > lo else np.zeros((H, W))


def edge_smooth_image(H, W, noise_std=5.0, seed=1):
    """Half a checkerboard-like field of cells 8-64 px with random step heights,
    half a 1/f-spectrum smooth field mapped to [0, 255], plus Gaussian noise."""
    rng = np.random.default_rng(seed)
    edge = _edge_field(H, W, rng)
    smooth = _smooth_field(H, W, rng)
    img = 0.5 * edge + 0.5 * smooth + rng.normal(0.0, noise_std, size=(H, W))
    return np.ascontiguousarray(np.clip(img, 0.0, 255.0), dtype=np.float32)


def weight_map(H, W, seed=3):
    """i.i.d. N(0, 1) weights (upstream gradient of a weighted-sum loss)."""
    return np.ascontiguousarray(np.random.default_rng(seed).normal(size=(H, W)), dtype=np.float32)


def checkerboard(n=150, cell=25, lo=0.0, hi=255.0):
    """Binary checkerboard, a stand-in for the sharp-edged test image of Table 1."""
    yy, xx = np.meshgrid(np.arange(n) // cell, np.arange(n) // cell, indexing="ij")
    return np.ascontiguousarray(np.where((yy + xx) % 2 == 0, lo, hi), dtype=np.float32)


def batch_specs(count=256, seed=4):
    """Uneven batch: per image H, W in {64..2048}, sigma_s in [2,16],
    sigma_r in [10,60], N in {4..16}, content seed 4+k."""
    rng = np.random.default_rng(seed)
    specs = []
    for k in range(count):
        specs.append({
            "H": int(rng.integers(64, 2049)), "W": int(rng.integers(64, 2049)),
            "sigma_s": float(rng.uniform(2.0, 16.0)), "sigma_r": float(rng.uniform(10.0, 60.0)),
            "N": int(rng.integers(4, 17)), "seed": seed + k,
        })
    return specs


def workload(name):
    """Named workloads: image and filter parameters."""
    if name == "rects512":          # 512x512, sigma_s=3, sigma_r=30, N=8
        return {"f": rects_image(512, 512, noise_std=10.0, seed=0),
                "sigma_s": 3.0, "sigma_r": 30.0, "N": 8}
    if name == "uhd":               # 3840x2160 edge+smooth field
        return {"f": edge_smooth_image(2160, 3840, noise_std=5.0, seed=1)}
    if name == "grad1024":          # 1024x1024, noise 20, weight map
        return {"f": rects_image(1024, 1024, noise_std=20.0, seed=2),
                "w": weight_map(1024, 1024, seed=3),
                "sigma_s": 5.0, "sigma_r": 25.0, "N": 10}
    if name == "8k":                # 8192x8192 edge+smooth field
        return {"f": edge_smooth_image(8192, 8192, noise_std=5.0, seed=5)}
    raise KeyError(name)
