"""FP64 CPU oracle of FORPDN, first-order spectral roughness penalty
denoising (test infrastructure only: imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs, never by the
product path).

The paper (Sec. 2.1) describes FORPDN in one sentence: a full-rank,
wavelet-based method, primarily for additive Gaussian noise, named for its
first-order spectral roughness penalty. The reading used here (kept
identical in the CUDA path):

1. ``sigma_b`` by the regression noise estimate of the HyRes stage
   (``oracle.hyres.noise_est_regression`` on the Gram matrix).
2. Every band image is padded (whole-sample symmetric, as in HyRes) and
   transformed by the L-level periodic db2 DWT (Mallat layout).
3. The coefficient positions fall into L + 1 groups: the detail positions
   of level l (l = 1..L) and the final LL band (group 0, as in
   ``oracle.hyres.level_map``). At each position the p band coefficients
   form a spectrum c.
4. Per group, with C the N_g x p matrix of its spectra (one row per
   position), the penalised least-squares estimate
   ``F = argmin 1/2 ||C - F||^2 + lam/2 ||F D^T||^2 = C (I + lam D^T D)^-1``,
   D the (p-1) x p first-difference operator along the bands (the
   first-order spectral roughness).
5. ``lam_g`` is the first minimiser over the grid ``lam_0 = 0``,
   ``lam_m = 10^(-3 + 7 (m - 1) / (K - 2))`` (m = 1..K-1) of Stein's unbiased
   risk estimate of the linear estimator S = (I + lam D^T D)^-1 under
   independent band noise of variances sigma_b^2:
   ``SURE_g(lam) = ||C S - C||^2 + 2 N_g sum_b sigma_b^2 S_bb - N_g sum_b sigma_b^2``.
6. The estimate is the inverse DWT of the smoothed coefficients, cropped.

The oracle evaluates step 4 and the SURE of step 5 from their definitions
(matrix inverse, traces); the CUDA path diagonalises D^T D by the DCT and
solves the tridiagonal systems directly.
"""

from __future__ import annotations

import numpy as np

from .hyres import dwt2, gram, idwt2, level_map, noise_est_regression, pad_symmetric, padded_shape


def diff_operator(p):
    """The (p-1) x p first-difference matrix: (D x)_b = x_{b+1} - x_b."""
    D = np.zeros((p - 1, p))
    for b in range(p - 1):
        D[b, b] = -1.0
        D[b, b + 1] = 1.0
    return D


def forpdn_lambda_grid(K):
    """lam_0 = 0, then K - 1 points spaced evenly in log10 from 1e-3 to 1e4."""
    lams = np.zeros(K)
    if K > 1:
        lams[1:] = 10.0 ** (-3.0 + 7.0 * np.arange(K - 1) / max(K - 2, 1))
    return lams


def smoother(p, lam):
    """S = (I + lam D^T D)^-1 (step 4)."""
    D = diff_operator(p)
    return np.linalg.inv(np.eye(p) + lam * (D.T @ D))


def sure_group(G, N, sigma2, lam):
    """Step 5 for one group from its Gram matrix G = C^T C (p x p) and its
    size N: ||C S - C||^2 = tr((S - I) G (S - I)), and the divergence term
    sum_b sigma_b^2 S_bb."""
    p = G.shape[0]
    S = smoother(p, lam)
    M = S - np.eye(p)
    return float(np.trace(M @ G @ M) + 2.0 * N * np.sum(sigma2 * np.diag(S)) - N * np.sum(sigma2))


def forpdn(Y, levels, n_lambda=64, sigma=None, k=None):
    """FORPDN on ``Y`` (``float[p][H][W]``). Returns a dict with ``X`` (float64
    cube), ``sigma``, the SURE table ``S`` [L + 1][K] (group 0 = LL), the
    chosen grid indices ``k`` [L + 1] and thresholds ``lam`` [L + 1]. ``k``
    given (one grid index per group) replaces the SURE choice: the estimate
    at another choice, for comparisons near ties."""
    Y = np.asarray(Y, dtype=np.float64)
    p, H, W = Y.shape
    n = H * W
    if sigma is None:
        sigma = noise_est_regression(gram(Y), n)
    sigma2 = np.asarray(sigma, dtype=np.float64) ** 2
    Hp, Wp = padded_shape(H, W, levels)
    C = np.stack([dwt2(pad_symmetric(Y[b], Hp, Wp), levels) for b in range(p)])   # [p][Hp][Wp]
    lev = level_map(Hp, Wp, levels)
    lams = forpdn_lambda_grid(n_lambda)
    S_tab = np.zeros((levels + 1, n_lambda))
    k_sel = np.zeros(levels + 1, dtype=np.int64)
    F = np.empty_like(C)
    for g in range(levels + 1):
        mask = lev == g
        Cg = C[:, mask].T                      # N_g x p, one spectrum per row
        N = Cg.shape[0]
        G = Cg.T @ Cg
        for m, lam in enumerate(lams):
            S_tab[g, m] = sure_group(G, N, sigma2, lam)
        k_sel[g] = int(np.argmin(S_tab[g])) if k is None else int(k[g])   # first minimiser
        F[:, mask] = (Cg @ smoother(p, lams[k_sel[g]])).T
    X = np.stack([idwt2(F[b], levels)[:H, :W] for b in range(p)])
    return dict(X=X, sigma=np.asarray(sigma, dtype=np.float64), S=S_tab, k=k_sel,
                lam=lams[k_sel], C=C)
