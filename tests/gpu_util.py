"""Helpers for the GPU tests: device buffers and Morton matrices through the C ABI."""
import numpy as np

import fm_inputs


def lib_and_device():
    import torch

    import __graft_entry__  # noqa: F401  (puts the repo root on sys.path)
    from paper_1705_04807_gb300 import build
    build.build()
    import paper_1705_04807_gb300 as fm
    fm.lib()
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return fm, torch.device("cuda:0")


def to_dev(x: np.ndarray, dev):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x).view(np.int32)).to(dev)


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def grid_for(rows, cols, lt):
    """Smallest log2 grid so that (2^lg * T')^2 holds rows x cols."""
    T = 1 << lt
    lg = 0
    while (1 << lg) * T < max(rows, cols, 1):
        lg += 1
    return lg


class MortonMatrix:
    """A device Morton-hybrid matrix owned by a torch tensor."""

    def __init__(self, fm, dev, lg, lt, fill=None):
        import torch
        n = (1 << lg) << lt
        self.n, self.lg, self.lt = n, lg, lt
        self.t = torch.zeros(n * n, dtype=torch.int32, device=dev)
        self.m = fm.matrix(self.t, lg, lt)
        self.fm, self.dev = fm, dev
        if fill is not None:
            self.load(fill)

    def load(self, x: np.ndarray, row0=0, col0=0):
        """Writes the row-major host array x at (row0, col0) through the device
        layout kernel (full matrix: x must be placed in an n x n canvas)."""
        canvas = np.zeros((self.n, self.n), dtype=np.uint32)
        canvas[row0:row0 + x.shape[0], col0:col0 + x.shape[1]] = x
        src = to_dev(canvas, self.dev)
        self.fm.fm_layout_to_morton(src, self.n, self.n, self.n, self.m)
        return self

    def read(self, rows=None, cols=None) -> np.ndarray:
        import torch
        rows = self.n if rows is None else rows
        cols = self.n if cols is None else cols
        out = torch.empty((rows, cols), dtype=torch.int32, device=self.dev)
        self.fm.fm_layout_from_morton(self.m, rows, cols, out, cols)
        return to_host(out)

    def sub(self, row0, col0, rows, cols):
        return self.fm.sub(self.m, row0, col0, rows, cols)


def residues(seed, shape, p, stream=0):
    return fm_inputs.uniform_residues(seed, shape, p, stream)
