"""Autotuner for batched filtering, with a JSON cache.

Two choices are tuned:
  * the row-pass kernel of the tensor-core form (BF_OPT_TILE_W: 0 = Toeplitz operand in
    tensor memory, 64 / 128 / 256 = Toeplitz operand in shared memory with tiles of that
    width), per bucket (a = ceil(R / 16), C = N + 2, width class, storage precision): the
    candidates are timed on a small batch of synthetic images of that bucket, run as one
    graph, so the choice is the one with the best throughput when images share the GPU.  The
    three widths give identical results; kernel 0 sums the same products in another order;
  * the number of concurrent graph branches of a batch, per batch composition (no effect on
    any result).
The cache maps "<device name>" -> {"tile_w": {bucket: width}, "branches": {signature: k}}
and is written after every new measurement.  `measure` can be replaced (tests use a fake
timer) and is called as measure(kind, **params) -> milliseconds.
"""
import json
import os
import threading

TILE_WIDTHS = (0, 64, 128, 256)
BRANCH_COUNTS = (1, 2, 4, 8, 16)
WIDTH_CLASSES = ((192, 128), (640, 512), (None, 1536))   # (upper bound of W, representative W)


def default_cache_path():
    return os.environ.get("BFGC_AUTOTUNE_CACHE",
                          os.path.join(os.path.expanduser("~"), ".cache", "bfgc", "autotune.json"))


def width_class(W):
    for i, (hi, _) in enumerate(WIDTH_CLASSES):
        if hi is None or W <= hi:
            return i
    return len(WIDTH_CLASSES) - 1


def tile_bucket(R, C, W, precision):
    a = max(1, (int(R) + 15) // 16)
    return f"{precision}/a{a}/C{int(C)}/w{width_class(W)}"


class Autotuner:
    def __init__(self, path=None, device_name=None, measure=None, reps=3):
        self.path = default_cache_path() if path is None else path
        self._device = device_name
        self.measure = self._measure_gpu if measure is None else measure
        self.reps = reps
        self._lock = threading.Lock()
        self._cache = self._load()
        self._images = {}                        # synthetic timing images by width

    # ---- cache
    @property
    def device(self):
        if self._device is None:
            import torch
            self._device = torch.cuda.get_device_name() if torch.cuda.is_available() else "cpu"
        return self._device

    def _load(self):
        try:
            with open(self.path) as fh:
                data = json.load(fh)
            return data if isinstance(data, dict) else {}
        except (OSError, ValueError):
            return {}

    def _entry(self):
        e = self._cache.setdefault(self.device, {})
        e.setdefault("tile_w", {})
        e.setdefault("branches", {})
        return e

    def save(self):
        d = os.path.dirname(self.path)
        if d:
            os.makedirs(d, exist_ok=True)
        tmp = self.path + f".tmp{os.getpid()}"
        with open(tmp, "w") as fh:
            json.dump(self._cache, fh, indent=1, sort_keys=True)
        os.replace(tmp, self.path)

    def cached(self):
        return json.loads(json.dumps(self._entry()))

    # ---- choices
    def tile_w(self, R, C, W, precision="bf16"):
        """BF_OPT_TILE_W for images of this bucket (widths 128 and 256 only when a <= 4)."""
        a = max(1, (int(R) + 15) // 16)
        cands = TILE_WIDTHS if a <= 4 else (0, 64)
        key = tile_bucket(R, C, W, precision)
        with self._lock:
            e = self._entry()
            if key not in e["tile_w"]:
                times = {tw: self.measure("tile_w", a=a, C=int(C), W=WIDTH_CLASSES[width_class(W)][1],
                                          precision=precision, tile_w=tw) for tw in cands}
                e["tile_w"][key] = min(cands, key=lambda tw: (times[tw], tw))
                self.save()
            return int(e["tile_w"][key])

    def branches(self, signature, run):
        """Branch count for a batch: run(k) -> milliseconds of one batch forward with k branches."""
        with self._lock:
            e = self._entry()
            if signature not in e["branches"]:
                times = {k: run(k) for k in BRANCH_COUNTS}
                e["branches"][signature] = min(BRANCH_COUNTS, key=lambda k: (times[k], k))
                self.save()
            return int(e["branches"][signature])

    # ---- measurement on the GPU
    def _measure_gpu(self, kind, a, C, W, precision, tile_w):
        """Milliseconds per image of a graph of 8 synthetic images of the bucket (H = 256)."""
        import torch

        from . import bfgc as B
        from .batch import GCBatch
        from .synth import edge_smooth_image
        assert kind == "tile_w"
        sigma_s = 16.0 * a / 3.0                 # R = 16 a, the bucket's largest radius
        specs = [{"H": 256, "W": W, "sigma_s": sigma_s, "sigma_r": 30.0, "N": C - 2, "tile_w": tile_w}
                 for _ in range(8)]
        batch = GCBatch(specs, form="fused_tc", precision=precision, branches=4)
        if W not in self._images:
            self._images[W] = [torch.from_numpy(edge_smooth_image(256, W, seed=100 + i)).cuda() for i in range(8)]
        fs = self._images[W]
        outs = [torch.empty_like(f) for f in fs]
        s = torch.cuda.current_stream()
        B.bf_gc_batch_forward(batch.handle, fs, outs, batch.ws, s)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        for _ in range(self.reps):
            B.bf_gc_batch_forward(batch.handle, fs, outs, batch.ws, s)
        e1.record(s)
        e1.synchronize()
        return e0.elapsed_time(e1) / (self.reps * len(fs))

