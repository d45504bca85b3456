"""FP64 CPU oracle of the HyRes hot path (test infrastructure only).

HyRes is the paper's automatic, parameter-free, low-rank, wavelet-based
denoiser for Gaussian noise (Sec. 2.1); the paper defers its internals to the
cited HyRes source. The stages written out here, in the order they run, are:

1. Gram matrix ``R = Y^T Y`` of the ``n x p`` pixel-by-band matrix.
2. Per-band noise level by multiple regression of each band on all the others
   (the HySime-style estimator the paper ships, Sec. 2.1).
3. Band whitening by those noise levels.
4. Eigendecomposition of the whitened Gram matrix (the spectral subspace of
   the low-rank model, Sec. 2.1 "low-rank").
5. Projection of the whitened cube onto the leading ``r_max`` eigenvectors.
6. Per-component 2D orthogonal Daubechies (db2) DWT (Sec. 2.1 "wavelet-based").
7. Stein's unbiased risk estimate (SURE) of soft-thresholding each component,
   on a grid of thresholds, and of dropping it.
8. Choice of rank r and threshold lambda minimising the total SURE (what makes
   the method "parameter-free", Sec. 2.1).
9. Soft-thresholding of the detail coefficients and the inverse DWT.
10. Back-projection to the band space and un-whitening.

Readings where the paper is silent (kept identical in the CUDA path):
periodic DWT boundary; whole-sample symmetric padding at the bottom/right to
multiples of 2**L, cropped after the inverse transform; the LL band is never
thresholded (thresholded too as a variant); one lambda shared by all kept
components (one per component as a variant); lambda grid
``k * sqrt(2 ln N) / (K - 1)``; ties go to the smallest rank, then the smallest
lambda; regression without intercept or ridge; uncentred Gram matrix.

Everything is plain float64 numpy. The input cube is float32 and is upcast
once; the oracle never reads anything produced by the CUDA path.
"""

from __future__ import annotations

import numpy as np


# --------------------------------------------------------------------------
# Wavelet filters and transforms (stage 6 and its inverse in stage 9)
# --------------------------------------------------------------------------

def db2_filters():
    """Daubechies' orthonormal 4-tap filter pair (two vanishing moments).

    Low-pass ``h = (1+s3, 3+s3, 3-s3, 1-s3) / (4 sqrt 2)`` with ``s3 = sqrt 3``
    (the closed form of the db2 scaling filter); high-pass is the quadrature
    mirror ``g_m = (-1)^m h_{3-m}``. Sec. 2.1 calls HyRes "wavelet-based"; db2
    is the orthogonal Daubechies wavelet this implementation uses.
    """
    s3 = np.sqrt(3.0)
    h = np.array([1.0 + s3, 3.0 + s3, 3.0 - s3, 1.0 - s3]) / (4.0 * np.sqrt(2.0))
    g = np.array([(-1.0) ** m * h[3 - m] for m in range(4)])
    return h, g


def _analysis_last_axis(x, h, g):
    """One periodic analysis step along the last axis.

    ``a_k = sum_m h_m x[(2k+m) mod M]`` and ``d_k = sum_m g_m x[(2k+m) mod M]``
    for ``k = 0 .. M/2-1``; the output holds ``a`` then ``d``.
    """
    M = x.shape[-1]
    k = np.arange(M // 2)
    a = np.zeros(x.shape[:-1] + (M // 2,))
    d = np.zeros(x.shape[:-1] + (M // 2,))
    for m in range(4):
        xm = x[..., (2 * k + m) % M]
        a += h[m] * xm
        d += g[m] * xm
    return np.concatenate([a, d], axis=-1)


def _synthesis_last_axis(c, h, g):
    """Transpose of ``_analysis_last_axis``: scatter each ``a_k, d_k`` back
    through the same taps, ``x[(2k+m) mod M] += h_m a_k + g_m d_k``."""
    M = c.shape[-1]
    half = M // 2
    a = c[..., :half]
    d = c[..., half:]
    k = np.arange(half)
    x = np.zeros(c.shape)
    for m in range(4):
        # for one m the targets (2k+m) mod M are distinct, so += is exact
        x[..., (2 * k + m) % M] += h[m] * a + g[m] * d
    return x


def _dwt2_one_level(block, h, g):
    # rows (W axis) first, then columns (H axis); Mallat layout: LL top-left
    t = _analysis_last_axis(block, h, g)
    t = np.swapaxes(_analysis_last_axis(np.swapaxes(t, -1, -2), h, g), -1, -2)
    return t


def _idwt2_one_level(block, h, g):
    t = np.swapaxes(_synthesis_last_axis(np.swapaxes(block, -1, -2), h, g), -1, -2)
    return _synthesis_last_axis(t, h, g)


def dwt2(img, levels):
    """L-level separable periodic db2 analysis of ``img[..., Hp, Wp]``.

    Each level transforms the current LL block (top-left ``Hp>>l x Wp>>l``)
    in place, rows then columns, so the result is in Mallat layout. ``Hp`` and
    ``Wp`` must be multiples of ``2**levels``.
    """
    h, g = db2_filters()
    C = np.array(img, dtype=np.float64, copy=True)
    Hp, Wp = C.shape[-2:]
    if Hp % (1 << levels) or Wp % (1 << levels):
        raise ValueError("image sides must be multiples of 2**levels")
    for lev in range(levels):
        hl, wl = Hp >> lev, Wp >> lev
        C[..., :hl, :wl] = _dwt2_one_level(C[..., :hl, :wl], h, g)
    return C


def idwt2(coef, levels):
    """Inverse of ``dwt2``: the exact transpose, coarsest level first."""
    h, g = db2_filters()
    X = np.array(coef, dtype=np.float64, copy=True)
    Hp, Wp = X.shape[-2:]
    for lev in reversed(range(levels)):
        hl, wl = Hp >> lev, Wp >> lev
        X[..., :hl, :wl] = _idwt2_one_level(X[..., :hl, :wl], h, g)
    return X


def padded_shape(H, W, levels):
    """Sides rounded up to multiples of ``2**levels``."""
    q = 1 << levels
    return -(-H // q) * q, -(-W // q) * q


def pad_symmetric(img, Hp, Wp):
    """Whole-sample symmetric extension at the bottom/right only:
    ``x[M + j] = x[M - 2 - j]`` (the edge sample is not repeated)."""
    H, W = img.shape[-2:]
    if Hp - H > H - 1 or Wp - W > W - 1:
        raise ValueError("padding longer than the image")
    pad = [(0, 0)] * (img.ndim - 2) + [(0, Hp - H), (0, Wp - W)]
    return np.pad(np.asarray(img, dtype=np.float64), pad, mode="reflect")


# --------------------------------------------------------------------------
# Stages 1-4: Gram matrix, noise estimation, whitening, eigendecomposition
# --------------------------------------------------------------------------

def gram(Y):
    """Stage 1: uncentred Gram matrix ``R = Y^T Y`` of the ``n x p`` matrix
    whose rows are pixels and columns are bands (input ``float[p][H][W]``)."""
    p = Y.shape[0]
    Yf = np.asarray(Y, dtype=np.float64).reshape(p, -1)
    return Yf @ Yf.T


def noise_est_regression(R, n):
    """Stage 2, as the method states it: regress band b on all other bands
    (least squares, no intercept) and take the residual power per pixel.

    The normal equations are sliced from ``R``:
    ``R[-b,-b] beta = R[-b,b]``, and
    ``sigma_b^2 = (R[b,b] - R[b,-b] beta) / n`` is the residual sum of squares
    over n. Returns ``sigma`` (float64[p]).
    """
    p = R.shape[0]
    sig2 = np.empty(p)
    for b in range(p):
        idx = np.array([j for j in range(p) if j != b])
        beta = np.linalg.solve(R[np.ix_(idx, idx)], R[idx, b])
        sig2[b] = (R[b, b] - R[b, idx] @ beta) / n
    return np.sqrt(sig2)


def noise_est_schur(R, n):
    """The same residual power through the Schur complement:
    ``sigma_b^2 = 1 / (n [R^-1]_bb)``."""
    return np.sqrt(1.0 / (n * np.diag(np.linalg.inv(R))))


def noise_est_lstsq(Y):
    """The same regression solved on the data matrix itself (QR/SVD based
    ``lstsq``), without forming ``R``; used only to pin the other two."""
    p = Y.shape[0]
    Yf = np.asarray(Y, dtype=np.float64).reshape(p, -1).T  # n x p
    n = Yf.shape[0]
    sig2 = np.empty(p)
    for b in range(p):
        others = np.delete(Yf, b, axis=1)
        beta, *_ = np.linalg.lstsq(others, Yf[:, b], rcond=None)
        res = Yf[:, b] - others @ beta
        sig2[b] = res @ res / n
    return np.sqrt(sig2)


def whiten_gram(R, sigma):
    """Stage 3 applied to the Gram matrix: ``R_w = D^-1 R D^-1`` with
    ``D = diag(sigma)``, i.e. the Gram matrix of the whitened cube
    ``Y D^-1``."""
    return R / np.outer(sigma, sigma)


def eig_desc(Rw):
    """Stage 4: symmetric eigendecomposition ``R_w = V diag(e) V^T`` with
    eigenvalues in descending order. Sign convention: the entry of largest
    magnitude of each eigenvector is made positive."""
    e, V = np.linalg.eigh(Rw)
    order = np.argsort(-e, kind="stable")
    e = e[order]
    V = V[:, order]
    piv = np.argmax(np.abs(V), axis=0)
    sgn = np.sign(V[piv, np.arange(V.shape[1])])
    sgn[sgn == 0] = 1.0
    return e, V * sgn


# --------------------------------------------------------------------------
# Stages 7-9: SURE, selection, soft threshold
# --------------------------------------------------------------------------

def soft_threshold(c, lam):
    """``sign(c) * max(|c| - lam, 0)``: the proximal map of ``lam * |x|``."""
    c = np.asarray(c, dtype=np.float64)
    return np.sign(c) * np.maximum(np.abs(c) - lam, 0.0)


def lambda_grid(N, K):
    """Threshold candidates ``lambda_k = k * sqrt(2 ln N) / (K - 1)``,
    ``k = 0..K-1``: a uniform grid up to the universal threshold for N
    unit-variance coefficients."""
    lam_max = np.sqrt(2.0 * np.log(N))
    return np.arange(K, dtype=np.float64) * (lam_max / (K - 1))


def _detail_mask(Hp, Wp, levels, threshold_ll=False):
    """Coefficients that are thresholded: the detail bands, and with
    ``threshold_ll`` the final LL band too."""
    m = np.ones((Hp, Wp), dtype=bool)
    if not threshold_ll:
        m[: Hp >> levels, : Wp >> levels] = False
    return m


def sure_table(C, levels, lams, threshold_ll=False):
    """Stage 7: SURE of each component ``C[i]`` (whitened, unit noise).

    For soft-thresholding the detail coefficients at ``lambda`` and keeping LL:
    ``S_i(lambda) = N - 2 #{detail: |c| <= lambda}
                    + sum_detail min(c^2, lambda^2)``
    (each LL coefficient, kept as is, contributes 1). With ``threshold_ll``
    (the variant that thresholds every coefficient) the counts and sums run
    over all N coefficients. For dropping the component (estimate zero):
    ``S_i(inf) = sum_all c^2 - N``. Evaluated by direct comparison against
    every candidate. Returns ``(S[r][K], S_inf[r])``.
    """
    r, Hp, Wp = C.shape
    N = Hp * Wp
    mask = _detail_mask(Hp, Wp, levels, threshold_ll)
    S = np.empty((r, len(lams)))
    S_inf = np.empty(r)
    for i in range(r):
        det = np.abs(C[i][mask])
        det2 = det * det
        for k, lam in enumerate(lams):
            inside = det <= lam
            S[i, k] = (N - 2.0 * np.count_nonzero(inside)
                       + np.sum(np.minimum(det2, lam * lam)))
        S_inf[i] = np.sum(C[i] * C[i]) - N
    return S, S_inf


def _level_groups(Hp, Wp, levels, threshold_ll):
    """Group (1..L) of every Mallat position for per-level thresholds: the
    detail bands of level l; the final LL band is group 0 (kept), or joins
    group L when it is thresholded too."""
    lev = level_map(Hp, Wp, levels)
    if threshold_ll:
        lev[lev == 0] = levels
    return lev


def sure_table_levels(C, levels, lams, threshold_ll=False):
    """Stage 7 split by level: for component ``i`` and group ``l`` (the
    detail coefficients of level l, plus the final LL band in group L with
    ``threshold_ll``), the SURE of soft-thresholding that group at
    ``lambda``: ``S_il(lambda) = N_l - 2 #{group: |c| <= lambda}
    + sum_group min(c^2, lambda^2)``, N_l the group's size. A component
    thresholded at ``lambda_l`` on group l has SURE ``n_kept + sum_l
    S_il(lambda_l)``, n_kept the number of coefficients kept as they are
    (the LL band unless ``threshold_ll``). Returns ``float[r][L][K]``."""
    r, Hp, Wp = C.shape
    lev = _level_groups(Hp, Wp, levels, threshold_ll)
    out = np.empty((r, levels, len(lams)))
    for i in range(r):
        for l in range(1, levels + 1):
            g = np.abs(C[i][lev == l])
            g2 = g * g
            for k, lam in enumerate(lams):
                out[i, l - 1, k] = (g.size - 2.0 * np.count_nonzero(g <= lam)
                                    + np.sum(np.minimum(g2, lam * lam)))
    return out


def sure_rank_lambda(S, S_inf):
    """Total SURE of keeping components ``1..r`` thresholded at ``lambda_k``
    and dropping ``r+1..r_max``: ``T[r-1][k] = sum_{i<=r} S_i(lambda_k) +
    sum_{r<i<=r_max} S_i(inf)``."""
    r_max = S.shape[0]
    head = np.cumsum(S, axis=0)
    tail = np.array([np.sum(S_inf[r + 1:]) for r in range(r_max)])
    return head + tail[:, None]


def select_rank_lambda(S, S_inf):
    """Stage 8: ``(r*, k*) = argmin T``; ties go to the smallest r, then the
    smallest k (row-major first minimum). Returns ``(r*, k*, T, gap)`` with
    ``gap`` the relative distance of the runner-up to the minimum."""
    T = sure_rank_lambda(S, S_inf)
    flat = int(np.argmin(T))
    r_star, k_star = divmod(flat, T.shape[1])
    vals = np.sort(T.ravel())
    gap = (vals[1] - vals[0]) / max(abs(vals[0]), 1e-300) if vals.size > 1 else np.inf
    return r_star + 1, k_star, T, gap


def select_rank_lambda_per_component(S, S_inf):
    """Stage 8 with one threshold per kept component (a reading the paper
    leaves open, Sec. 2.1): component ``i`` takes ``k_i``, the first
    minimiser of its own ``S_i(lambda_k)``; the rank minimises
    ``U[r-1] = sum_{i<=r} S_i(lambda_{k_i}) + sum_{r<i<=r_max} S_i(inf)``
    (first minimum). Returns ``(r*, k[r_max], U, gap)`` with ``gap`` the
    relative distance of the runner-up rank's ``U`` to the minimum."""
    S = np.asarray(S, dtype=np.float64)
    r_max = S.shape[0]
    k = np.argmin(S, axis=1)
    best = S[np.arange(r_max), k]
    U = np.array([np.sum(best[: r + 1]) + np.sum(S_inf[r + 1:]) for r in range(r_max)])
    r_star = int(np.argmin(U)) + 1
    vals = np.sort(U)
    gap = (vals[1] - vals[0]) / max(abs(vals[0]), 1e-300) if vals.size > 1 else np.inf
    return r_star, k, U, gap


def select_rank_lambda_per_level(S_lev, S_inf, n_kept):
    """Stage 8 with one threshold per kept component and level: group
    ``(i, l)`` takes ``k_il``, the first minimiser of ``S_il(lambda_k)``;
    component ``i`` then has SURE ``S*_i = n_kept + sum_l S_il(lambda_{k_il})``
    and the rank minimises ``U[r-1] = sum_{i<=r} S*_i + sum_{r<i<=r_max}
    S_i(inf)`` (first minimum). Returns ``(r*, k[r_max][L], U, gap)``."""
    S_lev = np.asarray(S_lev, dtype=np.float64)
    r_max = S_lev.shape[0]
    k = np.argmin(S_lev, axis=2)
    best = np.take_along_axis(S_lev, k[:, :, None], axis=2)[:, :, 0]
    comp = n_kept + best.sum(axis=1)
    U = np.array([np.sum(comp[: r + 1]) + np.sum(S_inf[r + 1:]) for r in range(r_max)])
    r_star = int(np.argmin(U)) + 1
    vals = np.sort(U)
    gap = (vals[1] - vals[0]) / max(abs(vals[0]), 1e-300) if vals.size > 1 else np.inf
    return r_star, k, U, gap


# --------------------------------------------------------------------------
# The whole path
# --------------------------------------------------------------------------

def hyres(Y, levels, r_max, n_lambda=64, *, sigma=None, V=None, rank=None,
          lam=None, lambda_mode="shared", threshold_ll=False):
    """Run stages 1-10 on ``Y`` (``float[p][H][W]``).

    Optional overrides (for checks of single stages): ``sigma`` (skip stage 2),
    ``V`` (``p x r_max`` basis, skip stage 4), ``rank`` and ``lam`` (skip
    stage 8). ``lambda_mode``: ``"shared"`` (one threshold for every kept
    component), ``"per_component"`` (``select_rank_lambda_per_component``;
    ``lam`` may then be a sequence of per-component thresholds) or
    ``"per_level"`` (``select_rank_lambda_per_level``; ``lam`` may then be a
    ``[rank][levels]`` table).
    ``threshold_ll``: the final LL band is thresholded (and counted in SURE)
    like the detail bands, instead of kept. Returns a
    dict with the estimate ``X`` (``float64[p][H][W]``) and every
    intermediate; ``lam_comp`` holds the threshold of each kept component
    (``[rank][levels]`` in the per-level mode).
    """
    if lambda_mode not in ("shared", "per_component", "per_level"):
        raise ValueError("lambda_mode must be 'shared', 'per_component' or 'per_level'")
    Y = np.asarray(Y)
    p, H, W = Y.shape
    n = H * W
    if not (1 <= r_max <= p):
        raise ValueError("need 1 <= r_max <= p")
    Yf = Y.reshape(p, n).astype(np.float64)
    R = Yf @ Yf.T                                               # stage 1
    if sigma is None:
        sigma = noise_est_regression(R, n)                      # stage 2
    sigma = np.asarray(sigma, dtype=np.float64)
    Rw = whiten_gram(R, sigma)                                  # stage 3
    evals, Vfull = eig_desc(Rw)                                 # stage 4
    if V is None:
        V = Vfull[:, :r_max]
    V = np.asarray(V, dtype=np.float64)
    Z = V.T @ (Yf / sigma[:, None])                             # stage 5
    Hp, Wp = padded_shape(H, W, levels)
    C = dwt2(pad_symmetric(Z.reshape(r_max, H, W), Hp, Wp), levels)  # stage 6
    N = Hp * Wp
    lams = lambda_grid(N, n_lambda)
    S, S_inf = sure_table(C, levels, lams, threshold_ll)        # stage 7
    r_star, k_star, T, gap = select_rank_lambda(S, S_inf)       # stage 8
    lam_star = lams[k_star]
    extra = {}
    if lambda_mode == "per_component":
        r_star, k_comp, U, gap = select_rank_lambda_per_component(S, S_inf)
        k_star, lam_star = int(k_comp[0]), lams[k_comp[0]]
        lam_comp = lams[k_comp[:r_star]]
        extra = dict(k_comp=k_comp, U=U)
    if lambda_mode == "per_level":
        n_kept = 0 if threshold_ll else (Hp >> levels) * (Wp >> levels)
        S_lev = sure_table_levels(C, levels, lams, threshold_ll)
        r_star, k_lev, U, gap = select_rank_lambda_per_level(S_lev, S_inf, n_kept)
        k_star, lam_star = int(k_lev[0, 0]), lams[k_lev[0, 0]]
        lam_comp = lams[k_lev[:r_star]]
        extra = dict(k_lev=k_lev, U=U, S_lev=S_lev)
    if rank is not None:
        r_star, k_star = int(rank), -1
        lam_star = lam
        shape = (r_star, levels) if lambda_mode == "per_level" else (r_star,)
        lam_comp = np.broadcast_to(np.asarray(lam, dtype=np.float64), shape)
    if lambda_mode == "shared":
        lam_star = float(lam_star)
        lam_comp = np.full(r_star, lam_star)
    # threshold of component i on level l (the LL band: group 0, kept, or
    # group L with threshold_ll)
    lam_il = np.asarray(lam_comp, dtype=np.float64)
    if lam_il.ndim == 1:
        lam_il = np.repeat(lam_il[:, None], levels, axis=1)
    groups = _level_groups(Hp, Wp, levels, threshold_ll)
    Ch = C[:r_star].copy()
    for i in range(r_star):                                     # stage 9
        for l in range(1, levels + 1):
            sel = groups == l
            Ch[i][sel] = soft_threshold(Ch[i][sel], lam_il[i, l - 1])
    Zh = idwt2(Ch, levels)[:, :H, :W].reshape(r_star, n)
    Xh = sigma[:, None] * (V[:, :r_star] @ Zh)                  # stage 10
    return dict(X=Xh.reshape(p, H, W), rank=r_star, k=k_star, lam=lam_star,
                lam_comp=np.array(lam_comp, dtype=np.float64),
                sigma=sigma, R=R, Rw=Rw, evals=evals, V=V, C=C, S=S,
                S_inf=S_inf, T=T, gap=gap, lams=lams, **extra)


# --------------------------------------------------------------------------
# Metrics (Sec. 3 reports PSNR and SAM without formulas; these are the
# standard definitions)
# --------------------------------------------------------------------------

def rel_l2(est, ref):
    """``||est - ref||_F / ||ref||_F`` in float64."""
    est = np.asarray(est, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    return float(np.linalg.norm((est - ref).ravel()) / np.linalg.norm(ref.ravel()))


def psnr(clean, est):
    """Mean over bands of ``10 log10(max(clean_b)^2 / MSE_b)``."""
    clean = np.asarray(clean, dtype=np.float64)
    est = np.asarray(est, dtype=np.float64)
    p = clean.shape[0]
    c = clean.reshape(p, -1)
    e = est.reshape(p, -1)
    mse = np.mean((c - e) ** 2, axis=1)
    return float(np.mean(10.0 * np.log10(np.max(c, axis=1) ** 2 / mse)))


def sam(clean, est):
    """Mean over pixels of the spectral angle ``arccos(<x, x^> / (|x| |x^|))``
    in radians."""
    p = clean.shape[0]
    c = np.asarray(clean, dtype=np.float64).reshape(p, -1)
    e = np.asarray(est, dtype=np.float64).reshape(p, -1)
    cos = np.sum(c * e, axis=0) / (np.linalg.norm(c, axis=0) * np.linalg.norm(e, axis=0))
    return float(np.mean(np.arccos(np.clip(cos, -1.0, 1.0))))


# --------------------------------------------------------------------------
# Differentiation form: learnable per-(component, level) threshold scales.
# The paper's package makes several conventional methods differentiable with
# PyTorch autograd and puts a trainable HyRes step in front of a DNN
# (Sec. 2.1, Sec. 2.2). Here the rank r* and base threshold lambda* are chosen
# by SURE at s = 1 and held fixed; the detail coefficients of component i at
# level l are thresholded at lambda* s[i][l].
# --------------------------------------------------------------------------

def level_map(Hp, Wp, levels):
    """Level (1..L) of every Mallat position; 0 for the final LL band."""
    lev = np.zeros((Hp, Wp), dtype=np.int64)
    for l in range(levels, 0, -1):
        hl, wl = Hp >> (l - 1), Wp >> (l - 1)
        blk = np.zeros((Hp, Wp), dtype=bool)
        blk[:hl, :wl] = True
        blk[: Hp >> l, : Wp >> l] = False
        lev[blk] = l
    return lev


def hyres_scaled(Y, levels, r_max, scale, n_lambda=64):
    """Forward of the differentiation form. ``scale`` is ``[p or r_max][L]``
    (rows >= r* unused). Returns the dict of ``hyres`` plus ``X_scaled``."""
    o = hyres(Y, levels, r_max, n_lambda)
    p, H, W = np.asarray(Y).shape
    r = o["rank"]
    C = o["C"][:r]
    Hp, Wp = C.shape[-2:]
    lev = level_map(Hp, Wp, levels)
    scale = np.asarray(scale, dtype=np.float64)
    Ch = C.copy()
    for i in range(r):
        for l in range(1, levels + 1):
            m = lev == l
            Ch[i][m] = soft_threshold(C[i][m], o["lam"] * scale[i, l - 1])
    Zh = idwt2(Ch, levels)[:, :H, :W].reshape(r, H * W)
    Xs = o["sigma"][:, None] * (o["V"][:, :r] @ Zh)
    o = dict(o)
    o["X_scaled"] = Xs.reshape(p, H, W)
    o["level_map"] = lev
    return o


def hyres_scaled_grad(Y, G, levels, r_max, scale, n_lambda=64):
    """Analytic gradient dL/ds of a loss with dL/dX_hat = G (``[p][H][W]``),
    by the adjoint chain: G -> V_r^T D G (transpose of the back-projection)
    -> zero-embed in H_p x W_p (transpose of the crop) -> DWT (the inverse DWT
    is orthogonal, so its transpose is the forward transform) -> times
    d soft(c, lam)/d lam = -sign(c) [|c| > lam] -> summed per (component,
    level) -> times lambda*. Returns ``dscale`` shaped like ``scale``."""
    o = hyres_scaled(Y, levels, r_max, scale, n_lambda)
    p, H, W = np.asarray(Y).shape
    r = o["rank"]
    Gf = np.asarray(G, dtype=np.float64).reshape(p, H * W)
    dZ = o["V"][:, :r].T @ (o["sigma"][:, None] * Gf)          # r x n
    Hp, Wp = o["C"].shape[-2:]
    dZp = np.zeros((r, Hp, Wp))
    dZp[:, :H, :W] = dZ.reshape(r, H, W)
    dC = dwt2(dZp, levels)
    lev = o["level_map"]
    C = o["C"][:r]
    scale = np.asarray(scale, dtype=np.float64)
    ds = np.zeros_like(scale)
    for i in range(r):
        for l in range(1, levels + 1):
            m = lev == l
            lam = o["lam"] * scale[i, l - 1]
            c = C[i][m]
            ds[i, l - 1] = o["lam"] * np.sum(dC[i][m] * (-np.sign(c)) * (np.abs(c) > lam))
    return ds, o


def mse_loss(Xh, Xc):
    """Mean squared error to the clean cube, ``||X_hat - X||^2 / numel``."""
    d = np.asarray(Xh, dtype=np.float64) - np.asarray(Xc, dtype=np.float64)
    return float(np.sum(d * d) / d.size)


def sure_loss_scaled(o, levels, scale):
    """SURE of the kept components with per-level thresholds lambda* s[i][l]:
    sum_i [N - sum_l (2 #{|c| <= lam_il} - sum min(c^2, lam_il^2))] over the
    detail coefficients of level l (LL kept). Returns (value, gradient) with
    the almost-everywhere gradient: d/dlam sum min(c^2, lam^2) =
    2 lam #{|c| > lam}, the count term being piecewise constant."""
    r = o["rank"]
    C = o["C"][:r]
    lev = o["level_map"]
    N = C.shape[-1] * C.shape[-2]
    scale = np.asarray(scale, dtype=np.float64)
    val = 0.0
    ds = np.zeros_like(scale)
    for i in range(r):
        val += N
        for l in range(1, levels + 1):
            m = lev == l
            lam = o["lam"] * scale[i, l - 1]
            c = np.abs(C[i][m])
            val += -2.0 * np.count_nonzero(c <= lam) + np.sum(np.minimum(c * c, lam * lam))
            ds[i, l - 1] = o["lam"] * 2.0 * lam * np.count_nonzero(c > lam)
    return float(val), ds
