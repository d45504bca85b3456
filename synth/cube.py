"""Seeded synthetic hyperspectral cubes.

The paper measures on the 2013 University of Houston cube with additive
Gaussian noise at a fixed input SNR (Sec. 3); that cube is not available here,
so these cubes stand in for it. They have the structure the low-rank wavelet
model expects of a real scene: a few smooth spectra (endmembers) mixed by
piecewise-smooth, sum-to-one abundance maps, plus band-dependent white
Gaussian noise.

Recipe (all random numbers from ``numpy.random.default_rng(seed)``, drawn in
the order written here, so a seed fixes the cube on every platform up to the
last-bit rounding of ``exp`` and ``matmul``):

* endmembers ``e_j(b) = 0.05 + sum_{q=1..3} a_q exp(-(b-mu_q)^2 / (2 w_q^2))``
  with ``a_q ~ U[0.2, 1]``, ``mu_q ~ U[0, p)``, ``w_q ~ U[p/20, p/5]``;
* abundances: ``m`` Voronoi seed points on the H x W grid; per pixel the logit
  of endmember j is ``4 * [pixel in region j]`` plus a smooth field made of 8
  Gaussian bumps (centre uniform, radius ``U[s/16, s/4]`` with
  ``s = min(H, W)``, amplitude ``U[-2, 2]``); abundances are the softmax over j;
* clean cube ``X = A E`` stored band-major (BSQ) as ``float32[p][H][W]``;
* noise ``sigma_b = s * u_b`` with ``u_b ~ U[1, spread]``, and ``s`` chosen so
  that the whole-cube SNR ``10 log10(||X||_F^2 / (n sum_b sigma_b^2))`` equals
  the requested value; an optional per-pixel map multiplies ``sigma_b``;
* noisy cube ``Y = X + sigma_b * N(0, 1)``, rounded once to float32.

Nothing in this module computes any stage of the denoiser.
"""

from __future__ import annotations

import numpy as np

# Named workloads. Sizes follow the paper's Houston scene (Sec. 3) for the
# full-size case and small cubes for the cases a CPU oracle finishes quickly.
CONFIGS = {
    # 64 x 64 px x 32 bands, 4 endmembers, 10 dB, db2 with 2 levels, r <= 8
    "c0": dict(H=64, W=64, p=32, m=4, snr_db=10.0, spread=4.0, seed=1,
               levels=2, r_max=8),
    # 349 x 1905 px x 144 bands (Houston 2013 shape), 12 endmembers, 10 dB,
    # sigma_b spread 4x, db2 with 5 levels, r <= 20
    "c1": dict(H=349, W=1905, p=144, m=12, snr_db=10.0, spread=4.0, seed=2,
               levels=5, r_max=20),
    # 128 x 128 px x 64 bands, one cube of the differentiable batch
    "c4": dict(H=128, W=128, p=64, m=8, snr_db=10.0, spread=4.0, seed=5,
               levels=4, r_max=16),
}


def cube_config(name: str) -> dict:
    """Return a copy of the named workload's parameters."""
    return dict(CONFIGS[name])


def _endmembers(rng: np.random.Generator, m: int, p: int) -> np.ndarray:
    b = np.arange(p, dtype=np.float64)
    E = np.full((m, p), 0.05)
    for j in range(m):
        a = rng.uniform(0.2, 1.0, size=3)
        mu = rng.uniform(0.0, p, size=3)
        w = rng.uniform(p / 20.0, p / 5.0, size=3)
        for q in range(3):
            E[j] += a[q] * np.exp(-((b - mu[q]) ** 2) / (2.0 * w[q] ** 2))
    return E


def _abundances(rng: np.random.Generator, m: int, H: int, W: int) -> np.ndarray:
    yy = np.arange(H, dtype=np.float64)
    xx = np.arange(W, dtype=np.float64)
    sy = rng.uniform(0, H, size=m)
    sx = rng.uniform(0, W, size=m)
    # nearest seed point (Voronoi region), computed separably per seed
    d2 = np.empty((m, H, W), dtype=np.float32)
    for j in range(m):
        d2[j] = ((yy[:, None] - sy[j]) ** 2 + (xx[None, :] - sx[j]) ** 2).astype(np.float32)
    region = np.argmin(d2, axis=0)
    del d2
    s = float(min(H, W))
    logits = np.empty((m, H, W), dtype=np.float64)
    for j in range(m):
        field = np.zeros((H, W), dtype=np.float64)
        cy = rng.uniform(0, H, size=8)
        cx = rng.uniform(0, W, size=8)
        rad = rng.uniform(s / 16.0, s / 4.0, size=8)
        amp = rng.uniform(-2.0, 2.0, size=8)
        for q in range(8):
            gy = np.exp(-((yy - cy[q]) ** 2) / (2.0 * rad[q] ** 2))
            gx = np.exp(-((xx - cx[q]) ** 2) / (2.0 * rad[q] ** 2))
            field += amp[q] * np.outer(gy, gx)
        logits[j] = 4.0 * (region == j) + field
    logits -= logits.max(axis=0, keepdims=True)
    A = np.exp(logits)
    A /= A.sum(axis=0, keepdims=True)
    return A  # (m, H, W), sums to one over m


def make_cube(H: int, W: int, p: int, m: int = 4, snr_db: float = 10.0,
              spread: float = 4.0, seed: int = 0,
              sigma_map: np.ndarray | None = None) -> dict:
    """Build one seeded synthetic cube.

    Returns a dict with
      ``Y``     noisy cube, ``float32[p][H][W]`` (BSQ, C-contiguous),
      ``X``     clean cube, ``float32[p][H][W]``,
      ``sigma`` the planted per-band noise standard deviations, ``float64[p]``
                (before ``sigma_map`` is applied),
      ``E``     endmember spectra ``float64[m][p]``.
    ``sigma_map`` (optional, ``float[H][W]``) multiplies the noise level of
    each pixel; the SNR target is then met by the unscaled ``sigma_b``.
    """
    if H < 1 or W < 1 or p < 1 or m < 1:
        raise ValueError("cube sizes must be positive")
    rng = np.random.default_rng(seed)
    E = _endmembers(rng, m, p)
    A = _abundances(rng, m, H, W)
    n = H * W
    # clean cube, band-major: X[b] = sum_j E[j, b] * A[j] (float64 for
    # cubes up to ~10^8 voxels, float32 beyond to bound host memory)
    if p * n <= 10 ** 8:
        X = (E.T @ A.reshape(m, n)).astype(np.float32).reshape(p, H, W)
    else:
        X = (E.T.astype(np.float32) @ A.reshape(m, n).astype(np.float32)).reshape(p, H, W)
    del A
    u = rng.uniform(1.0, spread, size=p)
    sig_pow = float(np.sum(X.astype(np.float64) ** 2))
    s2 = sig_pow / (n * float(np.sum(u ** 2)) * 10.0 ** (snr_db / 10.0))
    sigma = np.sqrt(s2) * u
    noise = rng.standard_normal((p, H, W), dtype=np.float32)
    noise *= sigma.astype(np.float32)[:, None, None]
    if sigma_map is not None:
        noise *= np.asarray(sigma_map, dtype=np.float32)[None, :, :]
    Y = X + noise
    del noise
    return dict(Y=np.ascontiguousarray(Y, dtype=np.float32),
                X=np.ascontiguousarray(X, dtype=np.float32),
                sigma=sigma, E=E)


def make_scene(H: int, W: int, p: int, table: np.ndarray, m: int = 12,
               snr_range: tuple = (5.0, 20.0), seed: int = 4) -> dict:
    """A scene for the sliding-window form: ``make_cube`` at 10 dB whole-cube
    SNR, with the noise of every window core scaled so that its own SNR is
    about ``U[snr_range]`` dB (the factor ``10^((10 - SNR_core) / 20)``
    multiplies sigma_b over the core). Returns the cube dict plus
    ``core_snr_db``."""
    rng = np.random.default_rng(seed + 1000)
    snr = rng.uniform(snr_range[0], snr_range[1], size=len(table))
    sigma_map = np.ones((H, W), dtype=np.float32)
    for (row, s_db) in zip(table, snr):
        cy, cx, ch, cw = (int(v) for v in row[4:8])
        sigma_map[cy:cy + ch, cx:cx + cw] = 10.0 ** ((10.0 - s_db) / 20.0)
    cube = make_cube(H, W, p, m=m, snr_db=10.0, seed=seed, sigma_map=sigma_map)
    cube["core_snr_db"] = snr
    return cube
