"""FP64 CPU oracle of HyMiNoR's sparse-noise stage (test infrastructure only:
imported by ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
legs, never by the product path).

The paper describes HyMiNoR in two sentences (Sec. 2.1): it is low-rank and
wavelet-based and builds on HyRes; after HyRes has removed the Gaussian noise,
the remaining sparse noise is removed by solving an l1-l1 optimisation problem
with a modified split-Bregman technique. It states neither the problem nor the
iteration. The reading used here (kept identical in the CUDA path):

1. ``G = HyRes(Y)`` (``oracle.hyres``), the Gaussian stage.
2. ``s = max |G|``; ``h = G / s``.
3. Per band image the l1-l1 problem
   ``min_x ||h_b - x||_1 + lam (||Dx x||_1 + ||Dy x||_1)``
   with ``Dx``, ``Dy`` the periodic forward differences along the image rows
   and columns: an l1 data term (the sparse residual) and an l1 penalty on
   the spatial differences (anisotropic total variation).
4. Split Bregman on the splitting ``A = h - x``, ``Bx = Dx x``, ``By = Dy x``
   with penalty ``mu`` on each constraint, from ``x = h`` and
   ``A = Bx = By = bA = bx = by = 0``, for ``iters`` iterations:

   * ``x``: the system ``(I + Dx^T Dx + Dy^T Dy) x = rhs``,
     ``rhs = (h - A + bA) + Dx^T (Bx - bx) + Dy^T (By - by)``, solved
     inexactly by two Jacobi sweeps from the current ``x`` (the system is
     ``5 x - (sum of the 4 neighbours) = rhs``; the modification of the
     split-Bregman iteration in this reading). An even number of sweeps
     matters: the Jacobi step has eigenvalue -4/5 on the checkerboard mode,
     which one sweep per outer iteration lets grow.
   * ``A = shrink(h - x + bA, 1/mu)``, ``bA += h - x - A``
   * ``Bx = shrink(Dx x + bx, lam/mu)``, ``bx += Dx x - Bx`` (same for y)

   (``shrink(v, t) = sign(v) max(|v| - t, 0)``).
5. ``X = s x``.

Defaults ``lam = 1`` (an isolated one-pixel spike of height h costs 4 lam h
in the penalty and h in the data term, so spikes go for lam > 1/4),
``mu = 10``, ``iters = 50``. Band images are independent problems.
"""

from __future__ import annotations

import numpy as np

from .hyres import hyres, soft_threshold


def dx(x):
    """Periodic forward difference along the last axis (image rows)."""
    return np.roll(x, -1, axis=-1) - x


def dy(x):
    """Periodic forward difference along the second-to-last axis (columns)."""
    return np.roll(x, -1, axis=-2) - x


def dxT(z):
    """Transpose of ``dx``: ``z[j-1] - z[j]`` (periodic)."""
    return np.roll(z, 1, axis=-1) - z


def dyT(z):
    """Transpose of ``dy``."""
    return np.roll(z, 1, axis=-2) - z


def tvl1_objective(h, x, lam):
    """``||h - x||_1 + lam (||Dx x||_1 + ||Dy x||_1)``, summed over the bands."""
    return float(np.sum(np.abs(h - x)) + lam * (np.sum(np.abs(dx(x))) + np.sum(np.abs(dy(x)))))


def tvl1_split_bregman(h, lam=1.0, mu=10.0, iters=50, sweeps=2):
    """Step 4 on band images ``h`` (``[p][H][W]`` or ``[H][W]``); returns ``x``."""
    h = np.asarray(h, dtype=np.float64)
    x = h.copy()
    A = np.zeros_like(h)
    bA = np.zeros_like(h)
    Bx = np.zeros_like(h)
    By = np.zeros_like(h)
    bx = np.zeros_like(h)
    by = np.zeros_like(h)
    for _ in range(iters):
        rhs = (h - A + bA) + dxT(Bx - bx) + dyT(By - by)
        for _s in range(sweeps):
            nb = (np.roll(x, 1, axis=-1) + np.roll(x, -1, axis=-1) +
                  np.roll(x, 1, axis=-2) + np.roll(x, -1, axis=-2))
            x = (rhs + nb) / 5.0
        A = soft_threshold(h - x + bA, 1.0 / mu)
        bA = bA + h - x - A
        gx, gy = dx(x), dy(x)
        Bx = soft_threshold(gx + bx, lam / mu)
        By = soft_threshold(gy + by, lam / mu)
        bx = bx + gx - Bx
        by = by + gy - By
    return x


def hyminor(Y, levels, r_max, n_lambda=64, lam=1.0, mu=10.0, iters=50, gaussian=None):
    """HyMiNoR on the cube ``Y`` (``float[p][H][W]``): HyRes, then the l1-l1
    stage on the normalised output. ``gaussian`` may pass a precomputed
    HyRes result (the dict of ``oracle.hyres``). Returns a dict with ``X``
    (float64 cube), ``G`` (the HyRes output) and ``s``."""
    g = gaussian if gaussian is not None else hyres(Y, levels, r_max, n_lambda)
    G = g["X"]
    s = float(np.max(np.abs(G)))
    if s == 0.0:
        return dict(X=np.zeros_like(G), G=G, s=s, hyres=g)
    x = tvl1_split_bregman(G / s, lam, mu, iters)
    return dict(X=s * x, G=G, s=s, hyres=g)
