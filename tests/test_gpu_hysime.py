"""GPU parity of HySime subspace identification (``hyde_hysime``) against
the FP64 oracle (``oracle/hysime.py``) on seeded cubes: p = 32 and p = 144,
10 to 30 dB.

The decisions must be identical: the dimension k and the kept candidates in
the same (ascending delta) order. The numbers are held to what float32
arithmetic on the GPU allows:

* delta of a kept candidate: |delta_gpu - delta_ora| <= 2e-4 |delta_ora| +
  2e-6 max|delta| (the Gram matrix carries ~1e-7 relative rounding, the
  inverse is refined in double, the eigenvectors are float32);
* every candidate's delta has the oracle's sign wherever the oracle's
  |delta| exceeds 1e-5 max|delta|;
* a kept eigenvector agrees with the oracle's up to sign within the angle a
  float32 eigensolver leaves at its eigenvalue gap g (relative to the
  largest eigenvalue): sin(angle) <= 2e-6 / g + 1e-6.

The 96 x 96 x 144 cube at 30 dB is chosen because its decision is close:
the last kept delta is -4.1e-5 of the largest and the first rejected one
+1.5e-5.
"""

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_cube

pytestmark = pytest.mark.gpu

CASES = [
    (64, 64, 32, 4, 10, 1),      # the 64 x 64 x 32 cube of the small workload
    (64, 64, 32, 5, 30, 3),
    (128, 128, 144, 8, 20, 21),
    (96, 96, 144, 6, 30, 22),    # close decision at the subspace boundary
]


@pytest.mark.parametrize("H,W,p,m,snr,seed", CASES)
def test_hysime_matches_oracle(hyde, H, W, p, m, snr, seed):
    c = make_cube(H, W, p, m=m, snr_db=snr, seed=seed)
    ref = O.hysime(c["Y"])
    got = hyde.hysime(torch.from_numpy(c["Y"]).cuda(), r_max=32)
    r = min(p, 32)
    assert got["status"] == 0
    assert got["k"] == ref["k"]
    assert not got["saturated"]
    idx = got["idx"].cpu().numpy()
    assert idx.tolist() == [int(i) for i in ref["idx"]]

    d_ref = ref["delta"][:r]
    d_got = got["delta"].cpu().numpy()
    scale = np.max(np.abs(d_ref))
    for i in idx:
        assert abs(d_got[i] - d_ref[i]) <= 2e-4 * abs(d_ref[i]) + 2e-6 * scale, i
    clear = np.abs(d_ref) > 1e-5 * scale
    assert np.all(np.sign(d_got[clear]) == np.sign(d_ref[clear]))

    ev = ref["evals"]
    ev_got = got["evals"].cpu().numpy()
    assert np.max(np.abs(ev_got - ev[:r])) <= 5e-6 * ev[0]
    V = got["V"].cpu().numpy()
    for i in idx:
        gap = min(abs(ev[i] - ev[i + 1]), abs(ev[i] - ev[i - 1]) if i > 0 else np.inf) / ev[0]
        v = V[:, i] / np.linalg.norm(V[:, i])
        w = ref["V"][:, i]
        sin = np.linalg.norm(v - (v @ w) * w)
        assert sin <= 2e-6 / gap + 1e-6, (i, sin, gap)
