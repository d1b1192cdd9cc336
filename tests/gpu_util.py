"""Helpers for the GPU tests: host<->device copies of the workload arrays and
one call into the C ABI through the Python binding."""
from __future__ import annotations

import numpy as np


def torch_cuda():
    import torch

    if not torch.cuda.is_available():
        raise RuntimeError("GPU tests need a CUDA device")
    return torch


def load_pip():
    from paper_2103_01216_gb300 import _build

    _build.build()
    import paper_2103_01216_gb300 as pip

    pip.lib()
    return pip


def to_dev(a: np.ndarray):
    torch = torch_cuda()
    if a.dtype == np.uint32:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int32))
    elif a.dtype == np.uint64:
        t = torch.from_numpy(np.ascontiguousarray(a).view(np.int64))
    else:
        raise TypeError(a.dtype)
    return t.cuda()


def from_dev(t, like: np.ndarray) -> np.ndarray:
    return t.cpu().numpy().view(like.dtype).reshape(like.shape)


def gpu_shuffle(pip, arr: np.ndarray, seed: int = 0, eps: float = 0.5, H: np.ndarray | None = None,
                with_stats: bool = False, **opts):
    """Copy arr to the GPU, shuffle it through the C ABI, return (host result, stats|None)."""
    torch = torch_cuda()
    A = to_dev(arr)
    Hd = to_dev(np.ascontiguousarray(H, dtype=np.uint32)) if H is not None else None
    st = torch.zeros(pip.STATS_BYTES, dtype=torch.uint8, device="cuda") if with_stats else None
    pip.shuffle(A, seed=seed, eps=eps, H=Hd, stats=st, **opts)
    pip.check()
    out = from_dev(A, arr)
    return out, (pip.read_stats(st) if with_stats else None)
