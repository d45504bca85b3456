"""GPU parity of WSRRR (``hyde_wsrrr``) against the FP64 oracle
(``oracle/wsrrr.py``): HyRes, then cyclic descent on the sparse
reduced-rank model (soft-thresholded wavelet coefficients, then the
orthogonal Procrustes basis, in double on the GPU).

Bars: HyRes's (rank, lambda) identical; the estimate within 1e-5 relative
L2 of the oracle's (1e-4 in the worst band); the features (component images
W2 B) within 1e-4 per component; with no iteration the output is HyRes's.
"""

import importlib

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_cube

pytestmark = pytest.mark.gpu

Wm = importlib.import_module("oracle.wsrrr")

CASES = [
    (64, 64, 32, 4, 1, 2, 8, 5),
    (77, 131, 24, 3, 31, 3, 6, 4),       # padded sides
    (96, 80, 144, 6, 3, 3, 12, 4),
    (40, 48, 20, 2, 7, 1, 4, 8),
]


def _run(hyde, c, L, r, iters, features=True):
    Y = torch.from_numpy(c["Y"]).cuda()
    X, info, F = hyde.wsrrr(Y, L, r, iters=iters, features=features)
    torch.cuda.synchronize()
    return X.cpu().numpy(), info, F.cpu().numpy()


@pytest.mark.parametrize("H,W,p,m,seed,L,r,iters", CASES)
def test_wsrrr_matches_oracle(hyde, H, W, p, m, seed, L, r, iters):
    c = make_cube(H, W, p, m=m, seed=seed)
    X, info, F = _run(hyde, c, L, r, iters)
    ref = Wm.wsrrr(c["Y"], L, r, iters=iters)
    assert info["status"] == 0
    assert info["rank"] == ref["rank"]
    err = O.rel_l2(X, ref["X"])
    band = max(O.rel_l2(X[b], ref["X"][b]) for b in range(p))
    ferr = max(O.rel_l2(F[i], ref["F"][i]) for i in range(ref["rank"]))
    print(f"{(H, W, p)} iters {iters}: rank {info['rank']}, rel-L2 {err:.2e}, worst band "
          f"{band:.2e}, features {ferr:.2e}, J {ref['J'][0]:.6g} -> {ref['J'][-1]:.6g}")
    assert err < 1e-5
    assert band < 1e-4
    assert ferr < 1e-4
    assert np.all(F[ref["rank"]:] == 0.0)


def test_wsrrr_without_iterations_is_hyres(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    Y = torch.from_numpy(c["Y"]).cuda()
    X0, info0 = hyde.wsrrr(Y, 2, 8, iters=0)
    Xh = hyde.hyres_denoise(Y, 2, 8)
    Xh = Xh[0] if isinstance(Xh, tuple) else Xh
    torch.cuda.synchronize()
    assert O.rel_l2(X0.cpu().numpy(), Xh.cpu().numpy()) < 1e-7


def test_wsrrr_full_cube(hyde):
    """The 349 x 1905 x 144 cube at five levels, three iterations."""
    c = make_cube(349, 1905, 144, m=12, seed=2)
    X, info, F = _run(hyde, c, 5, 20, 3)
    ref = Wm.wsrrr(c["Y"], 5, 20, iters=3)
    assert info["rank"] == ref["rank"]
    err = O.rel_l2(X, ref["X"])
    print(f"full cube: rank {info['rank']}, rel-L2 {err:.2e}")
    assert err < 1e-5


def test_wsrrr_rejects_unsupported_modes(hyde):
    Y = torch.zeros((8, 32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(hyde.HydeError):
        hyde.wsrrr(Y, 2, 4, iters=-1)
    with pytest.raises(hyde.HydeError):
        hyde.wsrrr(Y, 2, 4, precision=hyde.PREC_BF16X3)
