"""Seeded sliding-window tables for the batched (windowed) denoising form.

The paper denoises scenes too large for one pass by slicing them spatially
into tiles, denoising each tile and reassembling the result (Sec. 2.2.2). The
paper gives no tiling rule, so this module draws one: a seeded k-d split of
the scene into ``2**depth`` core rectangles (each split along the longer side
at a fraction ``U[0.3, 0.7]`` of its length, rounded to 8 px), redrawn until
every core side lies in ``[min_side, max_side]``. Each window is its core
grown by ``context`` pixels on every side that is not a scene border; the
output of a pixel is taken from the window whose core contains it, so every
pixel has exactly one source.

Table rows are ``int32[8]``: ``y0, x0, h, w`` of the window and
``cy0, cx0, ch, cw`` of its core, all in scene pixels.
"""

from __future__ import annotations

import numpy as np


def _split(rng, rect, depth, out):
    y0, x0, h, w = rect
    if depth == 0:
        out.append(rect)
        return
    if h >= w:
        cut = int(round(rng.uniform(0.3, 0.7) * h / 8.0)) * 8
        cut = min(max(cut, 8), h - 8)
        _split(rng, (y0, x0, cut, w), depth - 1, out)
        _split(rng, (y0 + cut, x0, h - cut, w), depth - 1, out)
    else:
        cut = int(round(rng.uniform(0.3, 0.7) * w / 8.0)) * 8
        cut = min(max(cut, 8), w - 8)
        _split(rng, (y0, x0, h, cut), depth - 1, out)
        _split(rng, (y0, x0 + cut, h, w - cut), depth - 1, out)


def make_window_table(H: int, W: int, depth: int = 9, context: int = 16,
                      min_side: int = 32, max_side: int = 224,
                      seed: int = 4, max_tries: int = 10000) -> np.ndarray:
    """Return an ``int32[2**depth][8]`` window table covering an H x W scene."""
    rng = np.random.default_rng(seed)
    for _ in range(max_tries):
        cores = []
        _split(rng, (0, 0, H, W), depth, cores)
        sides = np.array([(c[2], c[3]) for c in cores])
        if sides.min() >= min_side and sides.max() <= max_side:
            break
    else:
        raise RuntimeError("no window table met the side limits")
    rows = []
    for (cy, cx, ch, cw) in cores:
        y0 = max(cy - context, 0)
        x0 = max(cx - context, 0)
        y1 = min(cy + ch + context, H)
        x1 = min(cx + cw + context, W)
        rows.append((y0, x0, y1 - y0, x1 - x0, cy, cx, ch, cw))
    return np.asarray(rows, dtype=np.int32)
