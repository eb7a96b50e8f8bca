"""Animation with controllable flicker (Section 3.3).

The seed hierarchy is re-randomised per frame by changing the jitter seed:
with a fixed seed the chunk layout follows the guide (coherent), with a new
seed per frame the mosaic changes every frame, an effect that imitates
hand-coloured animation; a higher threshold gives larger chunks and so
stronger changes between frames.  `stylize_sequence` runs a sequence as one
batch launch; `flicker` measures the mean absolute RGBA change between
consecutive frames.
"""
from __future__ import annotations

import torch

from . import BatchFrame, stylize_batch

MODES = ("static", "per_frame")


def frame_seed(base_seed: int, t: int, mode: str) -> int:
    """Jitter seed of frame t: fixed ("static") or new every frame ("per_frame")."""
    if mode == "static":
        return base_seed & 0xFFFFFFFF
    if mode == "per_frame":
        return (base_seed + 0x9E3779B9 * (t + 1)) & 0xFFFFFFFF
    raise ValueError(f"mode must be one of {MODES}")


def stylize_sequence(guides, lut, style, levels: int, threshold: int, radius: int,
                     base_seed: int, mode: str = "per_frame", stream=None):
    """Stylises a list of target guides (frames of an animation) in one launch."""
    frames = [BatchFrame(g, lut, style, levels, threshold, frame_seed(base_seed, t, mode))
              for t, g in enumerate(guides)]
    return stylize_batch(frames, radius, stream=stream)


def flicker(frames) -> float:
    """Mean absolute RGBA difference between consecutive frames (0..255)."""
    diffs = [(b.int() - a.int()).abs().float().mean() for a, b in zip(frames, frames[1:])]
    return float(torch.stack(diffs).mean()) if diffs else 0.0
