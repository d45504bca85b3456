"""Seeded noise simulators: the noise kinds the paper's package provides as
utilities for testing denoisers (Sec. 2.1): additive Gaussian, non-i.i.d.
Gaussian, salt-and-pepper, dead lines and stripes. They make test inputs
only and compute no stage of any denoiser.

The paper names the kinds without defining them; the definitions used here
(all on a clean cube ``X``, ``float[p][H][W]``, with random numbers from
``numpy.random.default_rng(seed)`` drawn in the order written):

* ``gaussian``: ``X + sigma N(0, 1)`` with one sigma for every band, chosen so
  that ``10 log10(||X||^2 / (N sigma^2)) = snr_db`` (N voxels).
* ``noniid_gaussian``: ``sigma_b = s u_b``, ``u_b ~ U[1, spread]``, ``s`` set by
  the same whole-cube SNR.
* ``salt_and_pepper``: each voxel independently, with probability
  ``fraction``, set to the cube's minimum or maximum (equally likely).
* ``deadlines``: ``n_lines`` distinct columns, in a set of
  ``round(band_fraction * p)`` distinct bands, set to zero.
* ``stripes``: ``n_stripes`` distinct columns, in a set of
  ``round(band_fraction * p)`` distinct bands, shifted by one offset per
  (band, column) drawn from ``U[-amplitude, amplitude]`` times the band's
  standard deviation.

Each returns the noisy cube as float32 and a record of what it did.
"""

from __future__ import annotations

import numpy as np


def _as_cube(X):
    X = np.asarray(X, dtype=np.float64)
    if X.ndim != 3:
        raise ValueError("expected a cube float[p][H][W]")
    return X


def _sigma_for_snr(X, snr_db, weights):
    """Scale s with ``10 log10(||X||^2 / (H W sum_b (s w_b)^2)) = snr_db``."""
    p, H, W = X.shape
    power = np.sum(X * X)
    return np.sqrt(power / (H * W * np.sum(weights ** 2) * 10.0 ** (snr_db / 10.0)))


def gaussian(X, snr_db, seed=0):
    X = _as_cube(X)
    rng = np.random.default_rng(seed)
    w = np.ones(X.shape[0])
    s = _sigma_for_snr(X, snr_db, w)
    Y = X + s * rng.standard_normal(X.shape)
    return Y.astype(np.float32), dict(sigma=s * w)


def noniid_gaussian(X, snr_db, spread=4.0, seed=0):
    X = _as_cube(X)
    rng = np.random.default_rng(seed)
    u = rng.uniform(1.0, spread, size=X.shape[0])
    s = _sigma_for_snr(X, snr_db, u)
    Y = X + (s * u)[:, None, None] * rng.standard_normal(X.shape)
    return Y.astype(np.float32), dict(sigma=s * u)


def salt_and_pepper(X, fraction, seed=0):
    X = _as_cube(X)
    rng = np.random.default_rng(seed)
    hit = rng.random(X.shape) < fraction
    salt = rng.random(X.shape) < 0.5
    Y = X.copy()
    Y[hit & salt] = X.max()
    Y[hit & ~salt] = X.min()
    return Y.astype(np.float32), dict(mask=hit, salt=hit & salt)


def _bands(rng, p, band_fraction):
    nb = int(round(band_fraction * p))
    return np.sort(rng.choice(p, size=nb, replace=False))


def deadlines(X, n_lines, band_fraction=0.2, seed=0):
    X = _as_cube(X)
    rng = np.random.default_rng(seed)
    p, H, W = X.shape
    bands = _bands(rng, p, band_fraction)
    cols = np.sort(rng.choice(W, size=n_lines, replace=False))
    Y = X.copy()
    Y[np.ix_(bands, np.arange(H), cols)] = 0.0
    return Y.astype(np.float32), dict(bands=bands, cols=cols)


def stripes(X, n_stripes, band_fraction=0.2, amplitude=0.5, seed=0):
    X = _as_cube(X)
    rng = np.random.default_rng(seed)
    p, H, W = X.shape
    bands = _bands(rng, p, band_fraction)
    cols = np.sort(rng.choice(W, size=n_stripes, replace=False))
    offs = rng.uniform(-amplitude, amplitude, size=(len(bands), n_stripes))
    offs *= X[bands].reshape(len(bands), -1).std(axis=1)[:, None]
    Y = X.copy()
    for a, b in enumerate(bands):
        Y[b][:, cols] += offs[a][None, :]
    return Y.astype(np.float32), dict(bands=bands, cols=cols, offsets=offs)
