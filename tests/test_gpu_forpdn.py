"""GPU parity of FORPDN (``hyde_forpdn``) against the FP64 oracle
(``oracle/forpdn.py``): per wavelet-level group, the spectral smoothing
(I + lam D^T D)^-1 with lam chosen by SURE.

The GPU forms each group's SURE from float Gram matrices of the spectra
(summed in double) and the DCT diagonalisation of D^T D; the oracle from
the matrix definition in FP64. Bars: the SURE tables agree to 1e-5 of the
row's largest magnitude; the chosen grid index is the oracle's wherever the
oracle's minimum beats its runner-up by more than that, and otherwise is
a minimiser within it; the estimate matches the oracle run at the GPU's
choice to 1e-5 relative L2 (and per band to 1e-4).
"""

import importlib

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_cube

pytestmark = pytest.mark.gpu

F = importlib.import_module("oracle.forpdn")

CASES = [
    (64, 64, 32, 4, 1, 2),       # the 64 x 64 x 32 cube, two levels
    (77, 131, 24, 3, 31, 3),     # ragged sides (padded), p not a multiple of 4
    (96, 80, 144, 6, 3, 3),      # 144 bands
    (40, 41, 30, 2, 5, 1),       # one level, odd width
    (48, 40, 200, 5, 8, 2),      # 200 bands (the windows' band count)
]


def _check(c, L, got_X, info):
    Y = c["Y"]
    p = Y.shape[0]
    ref = F.forpdn(Y, L)
    sure = info["sure"].cpu().numpy()
    k_gpu = np.array(info["k"])
    assert info["status"] == 0
    for g in range(L + 1):
        row = ref["S"][g]
        tol = 1e-5 * np.max(np.abs(row))
        assert np.max(np.abs(sure[g] - row)) <= tol, (g, np.max(np.abs(sure[g] - row)), tol)
        order = np.argsort(row)
        clear = row[order[1]] - row[order[0]] > 2 * tol
        if clear:
            assert k_gpu[g] == ref["k"][g], (g, k_gpu[g], ref["k"][g])
        else:
            assert row[k_gpu[g]] <= row[ref["k"][g]] + 2 * tol
    at = ref if np.array_equal(k_gpu, ref["k"]) else F.forpdn(Y, L, k=k_gpu)
    X = got_X.cpu().numpy()
    err = O.rel_l2(X, at["X"])
    band = max(O.rel_l2(X[b], at["X"][b]) for b in range(p))
    print(f"{Y.shape}: k {k_gpu.tolist()} / {ref['k'].tolist()}, rel-L2 {err:.2e}, worst band {band:.2e}")
    assert err < 1e-5
    assert band < 1e-4
    return ref


@pytest.mark.parametrize("H,W,p,m,seed,L", CASES)
def test_forpdn_matches_oracle(hyde, H, W, p, m, seed, L):
    c = make_cube(H, W, p, m=m, seed=seed)
    X, info = hyde.forpdn(torch.from_numpy(c["Y"]).cuda(), L)
    torch.cuda.synchronize()
    ref = _check(c, L, X, info)
    # it denoises
    assert O.psnr(c["X"], ref["X"]) > O.psnr(c["X"], c["Y"]) + 3.0


def test_forpdn_full_cube(hyde):
    """The 349 x 1905 x 144 cube at five levels."""
    c = make_cube(349, 1905, 144, m=12, seed=2)
    X, info = hyde.forpdn(torch.from_numpy(c["Y"]).cuda(), 5)
    torch.cuda.synchronize()
    _check(c, 5, X, info)


def test_forpdn_rejects_bad_arguments(hyde):
    Y = torch.zeros((8, 16, 16), dtype=torch.float32, device="cuda")
    with pytest.raises(hyde.HydeError):
        hyde.forpdn(Y, 0)
    with pytest.raises(hyde.HydeError):
        hyde.forpdn(Y, 2, n_lambda=1)
    with pytest.raises(hyde.HydeError):
        hyde.forpdn(torch.zeros((300, 32, 32), dtype=torch.float32, device="cuda"), 2)
