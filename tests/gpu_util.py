"""Helpers for the GPU tests: device copies of uint16 arrays and buffers with
guard bands around a slice at a chosen unit offset (alignment control)."""
import numpy as np

CANARY = 0x5A5A


def torch_mod():
    import torch
    return torch


def to_dev(a: np.ndarray, device="cuda"):
    torch = torch_mod()
    return torch.from_numpy(np.ascontiguousarray(a).view(np.int16)).to(device)


def to_host(t) -> np.ndarray:
    return t.cpu().numpy().view(np.uint16)


class Guarded:
    """A device buffer holding `n` units at unit offset `off` (0..7 controls
    the misalignment), with canary units on both sides."""

    def __init__(self, n, off, fill=None, pad=64):
        torch = torch_mod()
        self.n, self.off, self.pad = n, off, pad
        total = pad + off + n + pad
        host = np.full(total, CANARY, dtype=np.uint16)
        if fill is not None:
            host[pad + off:pad + off + n] = fill
        self.base = to_dev(host)
        self.view = self.base[pad + off:pad + off + n]

    def get(self) -> np.ndarray:
        return to_host(self.view)

    def canaries_ok(self) -> bool:
        h = to_host(self.base)
        lo = h[:self.pad + self.off]
        hi = h[self.pad + self.off + self.n:]
        return bool(np.all(lo == CANARY) and np.all(hi == CANARY))


def first_diff(a, b, k=5):
    d = np.nonzero(a != b)[0]
    return d[:k].tolist(), int(d.size)
