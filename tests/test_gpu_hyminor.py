"""GPU parity of HyMiNoR (``hyde_hyminor``) against the FP64 oracle
(``oracle/hyminor.py``): HyRes, then the l1-l1 sparse-noise stage
(per-band anisotropic TV with an l1 data term, split Bregman with two
Jacobi sweeps per step), on seeded cubes with Gaussian noise plus
salt-and-pepper, stripe or dead-line noise from ``synth.noise``.

Bars: HyRes's (rank, lambda) choice identical; the output within 1e-4
relative L2 of the oracle's (HyRes matches to ~1e-6; a perturbation of the
l1-l1 stage's input grows by ~2x over 50 iterations in the oracle itself,
and float32 arithmetic on the compact state matches the FP64 oracle to
~1e-7); and the stage brings the estimate closer to the clean cube than
HyRes alone, as the oracle's does.
"""

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_cube
from synth import noise as N

pytestmark = pytest.mark.gpu


def _noisy(kind, c):
    if kind == "salt_and_pepper":
        return N.salt_and_pepper(c["Y"], 0.02, seed=2)[0]
    if kind == "stripes":
        return N.stripes(c["Y"], 8, band_fraction=0.3, amplitude=1.0, seed=2)[0]
    return N.deadlines(c["Y"], 6, band_fraction=0.3, seed=2)[0]


@pytest.mark.parametrize("H,W,p,m,L,r,kind,iters", [
    (64, 64, 32, 4, 2, 8, "salt_and_pepper", 50),
    (77, 131, 24, 3, 3, 6, "stripes", 50),      # ragged: partial tiles, periodic wrap
    (48, 48, 24, 3, 2, 6, "deadlines", 50),
    (40, 33, 16, 2, 2, 4, "salt_and_pepper", 1),  # the first iteration alone
    (20, 9, 8, 2, 1, 3, "stripes", 7),          # images smaller than a tile
])
def test_hyminor_matches_oracle(hyde, H, W, p, m, L, r, kind, iters):
    c = make_cube(H, W, p, m=m, seed=11)
    Yn = _noisy(kind, c)
    ref = O.hyminor(Yn, L, r, iters=iters)
    X, info = hyde.hyminor(torch.from_numpy(Yn).cuda(), L, r, iters=iters)
    torch.cuda.synchronize()
    got = X.cpu().numpy()
    assert info["status"] == 0
    g = ref["hyres"]
    assert (info["rank"], info["lambda_index"]) == (g["rank"], g["k"])
    err = O.rel_l2(got, ref["X"])
    assert err < 1e-4, err
    if iters >= 50:
        assert O.rel_l2(got, c["X"]) < O.rel_l2(ref["G"], c["X"])


def test_hyminor_full_cube(hyde):
    """The 349 x 1905 x 144 benchmark cube with 1 % salt-and-pepper noise on
    top of its Gaussian noise. Band images are independent l1-l1 problems, so
    the oracle's stage runs on four bands of its own HyRes output (scaled by
    the whole cube's max |G|) and those bands of the GPU output are compared
    with it, and with the clean cube."""
    c = make_cube(349, 1905, 144, m=12, seed=2)
    Yn = N.salt_and_pepper(c["Y"], 0.01, seed=3)[0]
    g = O.hyres(Yn, 5, 20)
    G = g["X"]
    s = float(np.max(np.abs(G)))
    bands = [0, 37, 101, 143]
    ref = s * O.tvl1_split_bregman(G[bands] / s, 1.0, 10.0, 50)
    X, info = hyde.hyminor(torch.from_numpy(Yn).cuda(), 5, 20)
    torch.cuda.synchronize()
    got = X.cpu().numpy()[bands]
    assert info["status"] == 0
    assert (info["rank"], info["lambda_index"]) == (g["rank"], g["k"])
    assert O.rel_l2(got, ref) < 1e-4, O.rel_l2(got, ref)
    assert O.rel_l2(got, c["X"][bands]) < O.rel_l2(G[bands], c["X"][bands])
