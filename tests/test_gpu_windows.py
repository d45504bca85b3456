"""GPU parity of the batched sliding-window form: every window is denoised
independently (own noise levels, subspace, rank, threshold) and the scene
takes each pixel from the window whose core holds it. Checked against the
FP64 oracle run window by window, eagerly and through one captured CUDA
graph, on a small scene in full and on the 2048 x 2048 x 200 scene with 512
uneven windows on a sample of windows."""

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_scene, make_window_table

pytestmark = pytest.mark.gpu


def _oracle_window(Y, row, L, r, K=64):
    y0, x0, h, w, cy, cx, ch, cw = (int(v) for v in row)
    o = O.hyres(Y[:, y0:y0 + h, x0:x0 + w], L, r, K)
    core = o["X"][:, cy - y0:cy - y0 + ch, cx - x0:cx - x0 + cw]
    return core, o


def test_windows_small_scene_full_parity(hyde):
    H, W, p, L, r = 192, 160, 24, 2, 6
    T = make_window_table(H, W, depth=4, context=8, min_side=16, max_side=96, seed=7)
    sc = make_scene(H, W, p, T, m=4, seed=9)
    Y = torch.from_numpy(sc["Y"]).cuda()
    win = hyde.HyResWindows(p, H, W, T, L, r, n_slots=5)
    X = win(Y)
    torch.cuda.synchronize()
    got = X.cpu().numpy()
    infos = win.infos()
    ref = np.zeros(sc["Y"].shape)
    for k, row in enumerate(T):
        core, o = _oracle_window(sc["Y"], row, L, r)
        y0, x0, h, w, cy, cx, ch, cw = (int(v) for v in row)
        ref[:, cy:cy + ch, cx:cx + cw] = core
        assert infos[k]["status"] == 0
        assert (infos[k]["rank"], infos[k]["lambda_index"]) == (o["rank"], o["k"]), k
    assert O.rel_l2(got, ref) < 1e-5
    # the captured graph reproduces the eager result
    X2 = torch.zeros_like(Y)
    win.capture(Y, X2)
    X2.zero_()
    win.replay()
    torch.cuda.synchronize()
    assert O.rel_l2(X2.cpu().numpy(), got) < 1e-6


def test_windows_full_scene_sampled(hyde):
    """2048 x 2048 x 200 scene, 512 windows of sides 48..256 with 16-px
    context, per-core SNR U[5, 20] dB, db2 with 3 levels, r <= 20; the whole
    scene through the captured graph. Every pixel of the scene must be
    written (the output starts as NaN) and finite; 18 windows are checked
    against the oracle (the smallest, the largest, window 16 and 15 drawn at
    random), one by one and together as a relative L2 error over their
    cores."""
    H = W = 2048
    p, L, r = 200, 3, 20
    T = make_window_table(H, W, depth=9, context=16, min_side=32, max_side=224, seed=4)
    sc = make_scene(H, W, p, T, m=12, seed=4)
    Y = torch.from_numpy(sc["Y"]).cuda()
    X = torch.zeros_like(Y)
    win = hyde.HyResWindows(p, H, W, T, L, r, n_slots=64)
    win.capture(Y, X)
    X.fill_(float("nan"))
    win.replay()
    torch.cuda.synchronize()
    infos = win.infos()
    assert all(i["status"] == 0 for i in infos)
    # the cores tile the scene: every pixel written, none left NaN or Inf
    assert bool(torch.isfinite(X).all())
    areas = T[:, 2] * T[:, 3]
    rng = np.random.default_rng(0)
    picks = {int(np.argmin(areas)), int(np.argmax(areas))}
    picks.add(16)   # 88 x 48 px x 200 bands: SURE keeps all r_max components
    rest = [k for k in range(len(T)) if k not in picks]
    picks |= set(int(k) for k in rng.choice(rest, size=15, replace=False))
    num = den = 0.0
    for k in sorted(picks):
        got, ref = _check_window(sc["Y"], T[k], L, r, infos[k], X, k)
        num += float(np.sum((got.astype(np.float64) - ref) ** 2))
        den += float(np.sum(ref ** 2))
    assert np.sqrt(num / den) < 1e-3


def _check_window(Y, row, L, r, info, X, k, tie_tol=1e-3):
    """Selection and reconstruction parity of one window.

    Where the selected rank reaches r_max the top-r_max subspace ends inside
    the cluster of near-equal noise eigenvalues; the split of that cluster
    into single components is then ill-determined (float32 against float64
    eigenvectors differ by a rotation inside it), and so is every
    per-component SURE term. Parity is then required up to a near-tie of the
    oracle's own SURE table (tie_tol relative, 1e-3 by default), and the reconstruction is
    compared with the oracle run at the GPU's choice, to the 1e-3 relative
    error the batched form is held to (1e-5 for every window whose rank is
    below r_max)."""
    core, o = _oracle_window(Y, row, L, r)
    y0, x0, h, w, cy, cx, ch, cw = (int(v) for v in row)
    got = X[:, cy:cy + ch, cx:cx + cw].cpu().numpy()
    choice = (info["rank"], info["lambda_index"])
    if choice == (o["rank"], o["k"]):
        ref = core
    else:
        Tm = o["T"]
        assert o["rank"] == r or o["gap"] < 1e-3, (k, choice, o["rank"], o["k"], o["gap"])
        assert Tm[choice[0] - 1, choice[1]] - Tm.min() <= tie_tol * abs(Tm.min()), k
        o2 = O.hyres(Y[:, y0:y0 + h, x0:x0 + w], L, r, rank=choice[0], lam=o["lams"][choice[1]])
        ref = o2["X"][:, cy - y0:cy - y0 + ch, cx - x0:cx - x0 + cw]
    tol = 1e-3 if choice[0] == r else 1e-5
    assert O.rel_l2(got, ref) < tol, (k, O.rel_l2(got, ref))
    return got, ref
