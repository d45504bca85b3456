"""FP64 CPU oracle of HySime subspace identification (test infrastructure
only: imported by ``tests/`` alone, never by the product path).

HySime is the signal-subspace identification that the paper ships for
FastHyDe and runs on GPUs (Sec. 2.1). Its published definition (Bioucas-Dias
and Nascimento, "Hyperspectral subspace identification", 2008) is followed
step by step:

1. Noise estimate: every band regressed on all the other bands (least
   squares, no intercept); the residuals are the noise estimate (the same
   estimator as stage 2 of the HyRes path).
2. Correlation matrices of the data, the noise and the signal (data minus
   noise), uncentred and normalised by the pixel count.
3. Eigenvectors of the signal correlation matrix, in descending eigenvalue
   order.
4. For each eigenvector e_i, the change in the mean squared error of
   projecting onto the subspace when e_i is included:
   ``delta_i = -e_i^T R_y e_i + 2 e_i^T R_n e_i`` (the projection error
   removed minus twice the noise power let through).
5. The subspace: the eigenvectors with negative delta, in ascending delta
   order; its dimension k is their number.

Readings where the definition leaves a choice: the correlation matrices are
uncentred (as the published code computes them); ties in delta keep the
eigenvalue order; delta exactly zero is not kept.
"""

from __future__ import annotations

import numpy as np

from .hyres import eig_desc


def hysime_noise(Yf):
    """Step 1 on the pixel-by-band matrix ``Yf`` (n x p, float64): the
    residual of each band's least-squares regression on the other bands,
    solved on the data (``lstsq``). Returns the n x p residual matrix."""
    n, p = Yf.shape
    W = np.empty_like(Yf)
    for b in range(p):
        others = np.delete(Yf, b, axis=1)
        beta, *_ = np.linalg.lstsq(others, Yf[:, b], rcond=None)
        W[:, b] = Yf[:, b] - others @ beta
    return W


def hysime_select(E, Ry, Rn):
    """Steps 4-5 for the eigenvectors ``E`` (p x m, columns): returns
    ``(k, idx, delta)``, ``idx`` the kept columns in ascending delta order
    (stable, so ties keep the column order)."""
    py = np.einsum("bi,bc,ci->i", E, Ry, E)
    pn = np.einsum("bi,bc,ci->i", E, Rn, E)
    delta = -py + 2.0 * pn
    order = np.argsort(delta, kind="stable")
    k = int(np.count_nonzero(delta < 0.0))
    return k, order[:k], delta


def hysime(Y):
    """HySime on the cube ``Y`` (``float[p][H][W]`` or ``[p][n]``). Returns
    a dict: ``k``; ``E`` (p x k, the subspace basis in ascending delta
    order); ``delta`` (per eigenvector, eigenvalue order); ``evals`` and
    ``V`` (all eigenpairs of R_x, descending); ``Ry``, ``Rn``, ``Rx``."""
    Y = np.asarray(Y)
    p = Y.shape[0]
    Yf = Y.reshape(p, -1).astype(np.float64).T          # n x p
    n = Yf.shape[0]
    if n < p:
        raise ValueError("need at least as many pixels as bands")
    W = hysime_noise(Yf)                                 # step 1
    X = Yf - W
    Ry = Yf.T @ Yf / n                                   # step 2
    Rn = W.T @ W / n
    Rx = X.T @ X / n
    evals, V = eig_desc(Rx)                              # step 3
    k, idx, delta = hysime_select(V, Ry, Rn)             # steps 4-5
    return dict(k=k, E=V[:, idx], idx=idx, delta=delta, evals=evals, V=V,
                Ry=Ry, Rn=Rn, Rx=Rx)
