"""CPU checks of the seeded noise simulators (test-input generators)."""

import numpy as np
import pytest

from synth import make_cube
from synth import noise as N


@pytest.fixture(scope="module")
def X():
    return make_cube(40, 56, 16, m=3, seed=30)["X"]


def _snr(X, Y):
    X = X.astype(np.float64)
    return 10.0 * np.log10(np.sum(X * X) / np.sum((Y.astype(np.float64) - X) ** 2))


@pytest.mark.parametrize("kind", ["gaussian", "noniid_gaussian"])
def test_gaussian_kinds_reach_the_snr(X, kind):
    Y, rec = getattr(N, kind)(X, 15.0, seed=1)
    assert Y.dtype == np.float32 and Y.shape == X.shape
    assert abs(_snr(X, Y) - 15.0) < 0.1
    if kind == "gaussian":
        assert np.all(rec["sigma"] == rec["sigma"][0])
    else:
        assert rec["sigma"].max() / rec["sigma"].min() > 1.5
        # per-band residual spread follows the per-band sigma
        res = (Y.astype(np.float64) - X).reshape(16, -1).std(axis=1)
        assert np.allclose(res / rec["sigma"], 1.0, atol=0.05)


def test_salt_and_pepper(X):
    Y, rec = N.salt_and_pepper(X, 0.05, seed=2)
    m = rec["mask"]
    assert abs(m.mean() - 0.05) < 0.005
    assert np.all(Y[rec["salt"]] == np.float32(X.max()))
    assert np.all(Y[m & ~rec["salt"]] == np.float32(X.min()))
    assert np.array_equal(Y[~m], X[~m])


def test_deadlines(X):
    Y, rec = N.deadlines(X, 5, band_fraction=0.25, seed=3)
    assert len(rec["bands"]) == 4 and len(rec["cols"]) == 5
    changed = Y != X
    for b in range(16):
        for c in range(56):
            dead = b in rec["bands"] and c in rec["cols"]
            assert np.all(Y[b, :, c] == 0.0) if dead else not changed[b, :, c].any()


def test_stripes(X):
    Y, rec = N.stripes(X, 6, band_fraction=0.5, amplitude=0.3, seed=4)
    D = Y.astype(np.float64) - X
    for a, b in enumerate(rec["bands"]):
        for j, c in enumerate(rec["cols"]):
            assert np.allclose(D[b, :, c], rec["offsets"][a, j], atol=1e-5)
    mask = np.zeros(D.shape, bool)
    mask[np.ix_(rec["bands"], np.arange(40), rec["cols"])] = True
    assert np.all(D[~mask] == 0.0)
    assert np.all(np.abs(rec["offsets"]) <= 0.3 * X.std(axis=(1, 2)).max() + 1e-12)


def test_simulators_are_seeded(X):
    for f, args in ((N.gaussian, (10.0,)), (N.salt_and_pepper, (0.1,)),
                    (N.stripes, (3,)), (N.deadlines, (3,))):
        assert np.array_equal(f(X, *args, seed=9)[0], f(X, *args, seed=9)[0])
        assert not np.array_equal(f(X, *args, seed=9)[0], f(X, *args, seed=10)[0])
