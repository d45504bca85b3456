"""The seeded input generators that the parity tests and the bench share
(no method arithmetic here): the sliding-window tables and the cubes.

Window tables: the cores tile the scene exactly once, each window is its core
grown by the context on every side that is not a scene border, core sides lie
in the requested range and on the 8-px grid of the k-d split, and the table
is a pure function of its seed. The benchmark scene's table (2048 x 2048, 512
windows) also meets the batched form's alignment (window x0 a multiple of 4).
Cubes: shapes and types, the planted endmember count is the rank of the
clean cube, the whole-cube SNR target, and the per-core noise scaling of a
scene.
"""

import numpy as np
import pytest

from synth import make_cube, make_scene, make_window_table


def _check_table(T, H, W, context, min_side, max_side):
    cover = np.zeros((H, W), dtype=np.int32)
    for row in T:
        y0, x0, h, w, cy, cx, ch, cw = (int(v) for v in row)
        cover[cy:cy + ch, cx:cx + cw] += 1
        assert min_side <= ch <= max_side and min_side <= cw <= max_side
        assert cy % 8 == 0 and cx % 8 == 0
        assert y0 == max(cy - context, 0) and x0 == max(cx - context, 0)
        assert y0 + h == min(cy + ch + context, H) and x0 + w == min(cx + cw + context, W)
    assert np.all(cover == 1)


@pytest.mark.parametrize("H,W,depth,ctx,mn,mx,seed", [
    (192, 160, 4, 8, 16, 96, 7),
    (128, 160, 3, 8, 24, 96, 3),
    (134, 124, 2, 8, 24, 96, 11),
    (2048, 2048, 9, 16, 32, 224, 4),
])
def test_window_table_tiles_the_scene(H, W, depth, ctx, mn, mx, seed):
    T = make_window_table(H, W, depth=depth, context=ctx, min_side=mn, max_side=mx, seed=seed)
    assert T.dtype == np.int32 and T.shape == (2 ** depth, 8)
    _check_table(T, H, W, ctx, mn, mx)
    assert np.array_equal(T, make_window_table(H, W, depth=depth, context=ctx, min_side=mn,
                                               max_side=mx, seed=seed))


def test_benchmark_scene_table_alignment_and_sides():
    T = make_window_table(2048, 2048, depth=9, context=16, min_side=32, max_side=224, seed=4)
    assert np.all(T[:, 1] % 4 == 0)          # window x0 on a 16-byte boundary
    win_sides = np.concatenate([T[:, 2], T[:, 3]])
    assert win_sides.min() >= 48 and win_sides.max() <= 256
    assert int(np.sum(T[:, 6].astype(np.int64) * T[:, 7])) == 2048 * 2048


def test_cube_rank_snr_and_types():
    c = make_cube(40, 36, 24, m=5, snr_db=10.0, seed=3)
    assert c["Y"].dtype == np.float32 and c["X"].dtype == np.float32
    assert c["Y"].shape == c["X"].shape == (24, 40, 36)
    assert c["Y"].flags["C_CONTIGUOUS"]
    s = np.linalg.svd(c["X"].reshape(24, -1).astype(np.float64), compute_uv=False)
    assert s[4] > 1e-3 * s[0] and s[5] < 1e-5 * s[0]     # rank m = 5
    noise = (c["Y"] - c["X"]).astype(np.float64)
    snr = 10 * np.log10(np.sum(c["X"].astype(np.float64) ** 2) / np.sum(noise ** 2))
    assert abs(snr - 10.0) < 0.5
    c2 = make_cube(40, 36, 24, m=5, snr_db=10.0, seed=3)
    assert np.array_equal(c["Y"], c2["Y"])


def test_scene_scales_noise_per_core():
    H = W = 64
    T = make_window_table(H, W, depth=2, context=8, min_side=16, max_side=48, seed=2)
    sc = make_scene(H, W, 16, T, m=3, seed=2)
    noise = (sc["Y"] - sc["X"]).astype(np.float64)
    ref = make_cube(H, W, 16, m=3, snr_db=10.0, seed=2)
    assert np.array_equal(sc["X"], ref["X"])
    # each core's noise is the unscaled draw times 10^((10 - SNR_core) / 20)
    base = (ref["Y"] - ref["X"]).astype(np.float64)
    for row, s_db in zip(T, sc["core_snr_db"]):
        cy, cx, ch, cw = (int(v) for v in row[4:8])
        f = 10.0 ** ((10.0 - s_db) / 20.0)
        a = noise[:, cy:cy + ch, cx:cx + cw]
        b = base[:, cy:cy + ch, cx:cx + cw]
        assert np.allclose(a, f * b, rtol=1e-4, atol=1e-6 * np.abs(b).max())
    assert np.all((sc["core_snr_db"] >= 5.0) & (sc["core_snr_db"] <= 20.0))
