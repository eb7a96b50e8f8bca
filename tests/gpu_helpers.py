"""Helpers shared by the GPU tests: numpy <-> device tensors and workload caches."""
import functools

import numpy as np
import torch

import synth


def to_dev(a: np.ndarray, dev) -> torch.Tensor:
    if a.dtype == np.uint16:
        a = a.view(np.int16)
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev)


def u32(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


@functools.lru_cache(maxsize=None)
def workload(name: str):
    if name == "256":
        return synth.workload_256()
    if name == "1080p":
        return synth.workload_1080p()
    if name == "4k":
        return synth.workload_4k_uv()
    raise KeyError(name)


def sample_pixels(seed: int, W: int, H: int, n: int, r: int = 0):
    """Random pixels plus the corners and points next to the frame borders."""
    rng = np.random.default_rng(seed)
    xs = list(rng.integers(0, W, n))
    ys = list(rng.integers(0, H, n))
    for (x, y) in [(0, 0), (W - 1, 0), (0, H - 1), (W - 1, H - 1), (W // 2, 0), (0, H // 2),
                   (min(W - 1, r), min(H - 1, r)), (W - 1 - min(W - 1, r), H // 3),
                   (63, 31), (64, 32), (min(W - 1, 65), min(H - 1, 33))]:
        xs.append(x)
        ys.append(y)
    return np.array(xs, dtype=np.int32), np.array(ys, dtype=np.int32)
