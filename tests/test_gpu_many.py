"""Several cubes at once (``hyde_hyres_denoise_many``): cubes of different
content over 3 workspace slots, each slot on its own stream. Every output
must equal the one-cube path bit for bit (the same kernels on the same
inputs; the slots share nothing), and every cube's info record its own
selection."""

import numpy as np
import pytest
import torch

from synth import make_cube

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("count,slots", [(5, 3), (2, 3), (4, 1), (6, 4)])
def test_many_cubes_equal_one_at_a_time(hyde, count, slots):
    H, W, p, L, r = 77, 131, 24, 3, 6
    cubes = [make_cube(H, W, p, m=3, seed=40 + k)["Y"] for k in range(count)]
    Ys = [torch.from_numpy(Y).cuda() for Y in cubes]
    Xs = [torch.full_like(Y, np.nan) for Y in Ys]
    many = hyde.HyResMany(p, H, W, L, r, slots=slots)
    many(Ys, Xs)
    torch.cuda.synchronize()
    one = hyde.HyRes(p, H, W, L, r)
    for k in range(count):
        ref = one(Ys[k]).clone()
        info = one.result_info()
        assert torch.equal(Xs[k], ref), k
        got = many.result_info(k)
        assert (got["status"], got["rank"], got["lambda_index"]) == \
            (info["status"], info["rank"], info["lambda_index"])


def test_many_rejects_bad_arguments(hyde):
    many = hyde.HyResMany(8, 32, 32, 2, 4, slots=2)
    Y = torch.zeros((8, 32, 32), dtype=torch.float32, device="cuda")
    with pytest.raises(ValueError):
        many([Y], [])
    with pytest.raises(hyde.HydeError):
        many([Y], [Y])          # in place is rejected by the library
