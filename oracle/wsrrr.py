"""FP64 CPU oracle of WSRRR, wavelet-based sparse reduced-rank regression
(test infrastructure only: imported by ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs, never by the
product path).

The paper (Sec. 2.1) says of WSRRR only that it is a low-rank,
wavelet-based method for Gaussian noise that can also extract features.
The reading used here (kept identical in the CUDA path):

* Whitened data on the padded domain, ``Yw = pad(Y_b / sigma_b)`` (the
  HyRes noise estimate and symmetric padding), as an N x p matrix (one row
  per padded pixel).
* The model ``Yw ~ W2 B V^T``: W2 the orthogonal L-level periodic db2
  synthesis applied to each of r component images, B their N x r wavelet
  coefficients (sparse), V a p x r matrix with orthonormal columns.
* The objective ``J(B, V) = 1/2 ||Yw - W2 B V^T||^2 + lam sum |B_detail|``
  (the final LL band is not penalised, as HyRes keeps it).
* Cyclic descent from HyRes's choice (V = its top-r* eigenvectors, r = r*,
  lam = lam*), each step an exact block minimisation:
  B <- soft(W2^T Yw V, lam) on the detail coefficients (LL kept), then
  V <- polar(Yw^T W2 B) (the orthogonal Procrustes solution: M = U S Q^T
  gives V = U Q^T). J never increases.
* After ``iters`` V-steps a last B-step; the estimate is
  ``sigma_b * (W2 B V^T)`` cropped; the r component images W2 B are the
  extracted features.

With ``iters = 0`` this is HyRes's estimate.
"""

from __future__ import annotations

import numpy as np

from .hyres import _level_groups, dwt2, hyres, idwt2, pad_symmetric, padded_shape, soft_threshold


def polar(M):
    """Orthonormal polar factor of M (p x r, full column rank): U Q^T from
    the thin SVD M = U S Q^T."""
    U, _, Qt = np.linalg.svd(M, full_matrices=False)
    return U @ Qt


def wsrrr(Y, levels, r_max, n_lambda=64, iters=10, hy=None):
    """WSRRR on ``Y`` (``float[p][H][W]``). ``hy`` may pass a precomputed
    ``oracle.hyres`` result. Returns a dict with ``X`` (float64 cube), ``V``,
    the features ``F`` (r component images, padded), ``J`` (the objective
    after every half-step), ``rank``, ``lam`` and ``sigma``."""
    Y = np.asarray(Y, dtype=np.float64)
    p, H, W = Y.shape
    g = hy if hy is not None else hyres(Y, levels, r_max, n_lambda)
    r, lam, sigma = int(g["rank"]), float(g["lam"]), np.asarray(g["sigma"], dtype=np.float64)
    V = np.array(g["V"][:, :r], dtype=np.float64)
    Hp, Wp = padded_shape(H, W, levels)
    N = Hp * Wp
    Yw = np.stack([pad_symmetric(Y[b] / sigma[b], Hp, Wp) for b in range(p)]).reshape(p, N)
    detail = _level_groups(Hp, Wp, levels, False) >= 1

    def bstep(V):
        C = dwt2((V.T @ Yw).reshape(r, Hp, Wp), levels)
        B = C.copy()
        B[:, detail] = soft_threshold(C[:, detail], lam)
        return B, idwt2(B, levels).reshape(r, N)

    def objective(V, B, F):
        return float(0.5 * np.sum((Yw - V @ F) ** 2) + lam * np.sum(np.abs(B[:, detail])))

    J = []
    for _ in range(iters):
        B, F = bstep(V)
        J.append(objective(V, B, F))
        V = polar(Yw @ F.T)
        J.append(objective(V, B, F))
    B, F = bstep(V)
    J.append(objective(V, B, F))
    Fc = F.reshape(r, Hp, Wp)[:, :H, :W].reshape(r, H * W)
    X = (sigma[:, None] * (V @ Fc)).reshape(p, H, W)
    return dict(X=X, V=V, F=F.reshape(r, Hp, Wp), B=B, J=np.array(J), rank=r, lam=lam,
                sigma=sigma, hyres=g)
