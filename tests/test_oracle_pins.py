"""Pins of the FP64 oracle against what the mathematics fixes.

Each test checks the oracle against something other than itself: closed
forms, an independent FFT route for the wavelet transform, brute force on tiny
inputs, power iteration, a QR/SVD least-squares route, a Monte Carlo
unbiasedness check of SURE, and special cases that reduce to a textbook
routine (truncated SVD). None of these need a GPU.
"""

import numpy as np
import pytest

import oracle as O
from synth import make_cube


# ---------------------------------------------------------------- db2 filters

def test_db2_filter_identities():
    h, g = O.db2_filters()
    # orthonormal scaling filter: unit norm, sum sqrt 2, double-shift orthogonal
    assert abs(np.sum(h * h) - 1.0) < 1e-15
    assert abs(np.sum(h) - np.sqrt(2.0)) < 1e-15
    assert abs(h[0] * h[2] + h[1] * h[3]) < 1e-16
    # wavelet filter: two vanishing moments, orthogonal to h at even shifts
    m = np.arange(4)
    assert abs(np.sum(g)) < 1e-15
    assert abs(np.sum(m * g)) < 1e-14
    assert abs(np.sum(h * g)) < 1e-16
    assert abs(g[0] * h[2] + g[1] * h[3]) < 1e-16
    assert abs(np.sum(g * g) - 1.0) < 1e-15


def test_db2_golden_taps():
    """Taps against the decimal values stored in tests/golden."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "db2_taps.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    gold_h = np.array([float(r[1]) for r in rows if r[0] == "h"])
    h, g = O.db2_filters()
    assert np.max(np.abs(h - gold_h)) < 1e-15


# ---------------------------------------------------------------- DWT

def _fft_analysis_1d(x, filt):
    """Periodic correlation y_j = sum_m f_m x[(j+m) mod M] by FFT, then the
    even samples: an independent route to one analysis step."""
    M = x.shape[-1]
    f = np.zeros(M)
    f[: len(filt)] = filt
    y = np.real(np.fft.ifft(np.fft.fft(x, axis=-1) * np.conj(np.fft.fft(f)), axis=-1))
    return y[..., 0::2]


def _fft_dwt2_one_level(img):
    h, g = O.db2_filters()
    rows_a = _fft_analysis_1d(img, h)
    rows_d = _fft_analysis_1d(img, g)
    out = np.zeros_like(img)
    H, W = img.shape
    for half, blk in ((0, rows_a), (1, rows_d)):
        ca = _fft_analysis_1d(blk.T, h).T   # column low-pass
        cd = _fft_analysis_1d(blk.T, g).T   # column high-pass
        out[: H // 2, half * W // 2:(half + 1) * W // 2] = ca
        out[H // 2:, half * W // 2:(half + 1) * W // 2] = cd
    return out


@pytest.mark.parametrize("H,W", [(8, 8), (16, 12), (6, 10), (32, 64)])
def test_dwt_one_level_matches_fft_route(H, W):
    rng = np.random.default_rng(H * 100 + W)
    x = rng.standard_normal((H, W))
    assert np.max(np.abs(O.dwt2(x, 1) - _fft_dwt2_one_level(x))) < 1e-12


def test_dwt_multilevel_matches_fft_route():
    rng = np.random.default_rng(7)
    x = rng.standard_normal((32, 48))
    ref = _fft_dwt2_one_level(x)
    ref[:16, :24] = _fft_dwt2_one_level(ref[:16, :24])
    ref[:8, :12] = _fft_dwt2_one_level(ref[:8, :12])
    assert np.max(np.abs(O.dwt2(x, 3) - ref)) < 1e-12


@pytest.mark.parametrize("shape,L", [((64, 64), 2), ((352, 96), 5), ((3, 40, 24), 3), ((16, 8), 3)])
def test_dwt_perfect_reconstruction_and_parseval(shape, L):
    rng = np.random.default_rng(sum(shape) + L)
    x = rng.standard_normal(shape) * 3.0 + 1.0
    c = O.dwt2(x, L)
    assert np.linalg.norm(O.idwt2(c, L) - x) / np.linalg.norm(x) < 1e-12
    assert abs(np.sum(c * c) - np.sum(x * x)) < 1e-12 * np.sum(x * x)


def test_dwt_matrix_is_orthogonal_brute_force():
    H, W, L = 8, 8, 2
    n = H * W
    M = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        M[:, j] = O.dwt2(e.reshape(H, W), L).ravel()
    assert np.max(np.abs(M.T @ M - np.eye(n))) < 1e-13
    Minv = np.zeros((n, n))
    for j in range(n):
        e = np.zeros(n)
        e[j] = 1.0
        Minv[:, j] = O.idwt2(e.reshape(H, W), L).ravel()
    assert np.max(np.abs(Minv - M.T)) < 1e-13   # synthesis is the transpose


def test_dwt_delta_gives_taps():
    """A delta at (0, 0) hits output k only through tap m = -2k mod M."""
    h, g = O.db2_filters()
    x = np.zeros((8, 8))
    x[0, 0] = 1.0
    c = O.dwt2(x, 1)
    # row 0 only gets taps at k=0 (m=0); wrap k=3 (2*3 + 2 = 8 = 0 mod 8) gets m=2
    assert abs(c[0, 0] - h[0] * h[0]) < 1e-15
    assert abs(c[0, 3] - h[0] * h[2]) < 1e-15
    assert abs(c[0, 4] - h[0] * g[0]) < 1e-15       # row detail, col low
    assert abs(c[4, 0] - g[0] * h[0]) < 1e-15       # col detail, row low
    assert abs(c[7, 7] - g[2] * g[2]) < 1e-15
    assert np.count_nonzero(np.abs(c) > 1e-15) == 16


def test_dwt_constant_and_ramp_have_no_detail():
    L = 3
    c = O.dwt2(np.full((32, 32), 2.5), L)
    det = c.copy()
    det[:4, :4] = 0
    assert np.max(np.abs(det)) < 1e-13
    # a linear ramp along W: row details vanish except where the filter wraps
    x = np.tile(np.arange(32.0), (16, 1))
    c1 = O.dwt2(x, 1)
    row_detail = c1[:8, 16:]
    assert np.max(np.abs(row_detail[:, :-1])) < 1e-12
    assert np.max(np.abs(row_detail[:, -1])) > 1.0


def test_symmetric_pad_and_shape():
    assert O.padded_shape(349, 1905, 5) == (352, 1920)
    assert O.padded_shape(64, 64, 2) == (64, 64)
    x = np.arange(5.0)[None, :] * np.ones((3, 1))
    xp = O.pad_symmetric(x, 4, 8)
    assert np.array_equal(xp[0], [0, 1, 2, 3, 4, 3, 2, 1])
    assert np.array_equal(xp[3], xp[1])


# ---------------------------------------------------------------- soft threshold

def test_soft_threshold_is_prox_of_l1():
    grid = np.linspace(-6, 6, 120001)
    for c in (-3.3, -0.4, 0.0, 0.7, 2.5):
        for lam in (0.0, 0.5, 1.0):
            obj = 0.5 * (grid - c) ** 2 + lam * np.abs(grid)
            assert abs(grid[np.argmin(obj)] - O.soft_threshold(c, lam)) < 2e-4
    c = np.linspace(-4, 4, 81)
    assert np.array_equal(O.soft_threshold(-c, 1.3), -O.soft_threshold(c, 1.3))
    assert np.array_equal(O.soft_threshold(c, 0.0), c)


# ---------------------------------------------------------------- eigen

def _power_deflation(A, iters=3000):
    A = A.copy()
    p = A.shape[0]
    vals, vecs = [], []
    rng = np.random.default_rng(0)
    for _ in range(p):
        v = rng.standard_normal(p)
        v /= np.linalg.norm(v)
        for _ in range(iters):
            w = A @ v
            v = w / np.linalg.norm(w)
        lam = v @ A @ v
        vals.append(lam)
        vecs.append(v)
        A = A - lam * np.outer(v, v)
    return np.array(vals), np.array(vecs).T


@pytest.mark.parametrize("p", [3, 4, 6, 8])
def test_eig_against_power_iteration(p):
    rng = np.random.default_rng(p)
    Q, _ = np.linalg.qr(rng.standard_normal((p, p)))
    lam = 10.0 * 0.6 ** np.arange(p)
    A = (Q * lam) @ Q.T
    e, V = O.eig_desc(A)
    pe, pv = _power_deflation(A)
    assert np.max(np.abs(e - pe)) < 1e-12 * lam[0]
    for i in range(p):
        assert abs(abs(V[:, i] @ pv[:, i]) - 1.0) < 1e-10
    assert np.max(np.abs((V * e) @ V.T - A)) < 1e-13 * lam[0]
    assert np.max(np.abs(V.T @ V - np.eye(p))) < 1e-13
    assert np.all(np.diff(e) <= 0)
    assert np.all(V[np.argmax(np.abs(V), axis=0), np.arange(p)] > 0)


# ---------------------------------------------------------------- noise estimate

def test_noise_routes_agree_c0():
    c = make_cube(64, 64, 32, m=4, seed=1)
    R = O.gram(c["Y"])
    s1 = O.noise_est_regression(R, 64 * 64)
    s2 = O.noise_est_schur(R, 64 * 64)
    s3 = O.noise_est_lstsq(c["Y"])
    assert np.max(np.abs(s1 / s2 - 1)) < 1e-10
    assert np.max(np.abs(s1 / s3 - 1)) < 1e-9


def test_noise_regression_exact_on_constructed_residual():
    """If y_b = Y_-b beta + e with e orthogonal to the regressors, the
    regression residual power is exactly |e|^2 / n."""
    rng = np.random.default_rng(3)
    n, p = 500, 6
    for b in range(p):
        others = rng.standard_normal((n, p - 1))
        q, _ = np.linalg.qr(others)
        e = rng.standard_normal(n)
        e -= q @ (q.T @ e)
        yb = others @ rng.standard_normal(p - 1) + e
        Y = np.insert(others, b, yb, axis=1).T.reshape(p, 20, 25)
        s = O.noise_est_regression(O.gram(Y), n)
        assert abs(s[b] ** 2 - (e @ e) / n) < 1e-10 * (e @ e) / n


def test_noise_recovers_planted_sigma():
    """Median relative error of the planted per-band sigma within 5 %.

    The regression has noisy regressors, so bands whose signal is poorly
    predicted by the others are biased upward (errors-in-variables); the
    estimate must never be below the truth by more than sampling error."""
    for (H, W, p, m, seed) in [(64, 64, 32, 4, 1), (128, 128, 64, 8, 5)]:
        c = make_cube(H, W, p, m=m, seed=seed)
        s = O.noise_est_regression(O.gram(c["Y"]), H * W)
        rel = s / c["sigma"] - 1.0
        assert np.median(np.abs(rel)) < 0.05
        assert rel.min() > -4.0 / np.sqrt(H * W) - 0.02


# ---------------------------------------------------------------- SURE

@pytest.mark.parametrize("threshold_ll", [False, True])
def test_sure_is_unbiased_monte_carlo(threshold_ll):
    """With the basis and noise levels fixed independently of the noise,
    SURE(r, lambda) is an unbiased estimate of the whitened squared error,
    with the LL band kept or thresholded too. 64 noise draws; every (r, k)
    cell within 4.5 standard errors and 90 % within 2.5."""
    H, W, p, L, K = 32, 32, 12, 2, 16
    base = make_cube(H, W, p, m=3, seed=11)
    Xc = base["X"].astype(np.float64)
    sigma = base["sigma"]
    Xw = Xc.reshape(p, -1) / sigma[:, None]
    _, V = O.eig_desc(Xw @ Xw.T)       # full p x p basis from the clean cube
    rng = np.random.default_rng(12345)
    lams = O.lambda_grid(H * W, K)
    det_mask = np.ones((H, W), bool)
    if not threshold_ll:
        det_mask[: H >> L, : W >> L] = False
    C_clean = O.dwt2((V.T @ Xw).reshape(p, H, W), L)
    sure_vals, loss_vals = [], []
    for _ in range(64):
        Yw = Xw + rng.standard_normal(Xw.shape)
        C = O.dwt2((V.T @ Yw).reshape(p, H, W), L)
        S, S_inf = O.sure_table(C, L, lams, threshold_ll)
        T = O.sure_rank_lambda(S, S_inf)
        loss = np.empty_like(T)
        for r in range(1, p + 1):
            for k, lam in enumerate(lams):
                Ch = C.copy()
                Ch[r:] = 0.0
                Ch[:r, det_mask] = O.soft_threshold(Ch[:r, det_mask], lam)
                loss[r - 1, k] = np.sum((Ch - C_clean) ** 2)
        sure_vals.append(T)
        loss_vals.append(loss)
    diff = np.array(sure_vals) - np.array(loss_vals)
    z = diff.mean(axis=0) / (diff.std(axis=0, ddof=1) / np.sqrt(diff.shape[0]))
    assert np.max(np.abs(z)) < 4.5
    assert np.mean(np.abs(z) < 2.5) > 0.9


def test_sure_single_component_closed_form():
    """Tiny hand case: LL = 1 coefficient, 3 detail coefficients."""
    C = np.zeros((1, 2, 2))
    C[0] = [[5.0, 0.5], [-2.0, 1.5]]
    S, S_inf = O.sure_table(C, 1, np.array([0.0, 1.0, 3.0]))
    # lam = 0: N - 2*0 + 0 = 4 (no detail coefficient is exactly 0)
    # lam = 1: 4 - 2*1 + (0.25 + 1 + 1) = 4.25
    # lam = 3: 4 - 2*3 + (0.25 + 4 + 2.25) = 4.5
    assert np.allclose(S[0], [4.0, 4.25, 4.5], atol=1e-15)
    assert abs(S_inf[0] - (25 + 0.25 + 4 + 2.25 - 4)) < 1e-14


def test_sure_threshold_all_closed_form():
    """The hand case above with the LL coefficient thresholded too."""
    C = np.zeros((1, 2, 2))
    C[0] = [[5.0, 0.5], [-2.0, 1.5]]
    S, S_inf = O.sure_table(C, 1, np.array([0.0, 1.0, 3.0]), threshold_ll=True)
    # lam = 1: 4 - 2*1 + (1 + 0.25 + 1 + 1) = 5.25
    # lam = 3: 4 - 2*3 + (9 + 0.25 + 4 + 2.25) = 13.5
    assert np.allclose(S[0], [4.0, 5.25, 13.5], atol=1e-15)
    assert abs(S_inf[0] - (25 + 0.25 + 4 + 2.25 - 4)) < 1e-14


@pytest.mark.parametrize("threshold_ll", [False, True])
def test_full_rank_residual_is_clipped_energy(threshold_ll):
    """At full rank on an unpadded cube (sides multiples of 2^L) the
    whitening, the eigenbasis and the DWT are invertible and the last two
    orthogonal, so the whitened residual energy of the estimate is the energy
    the soft threshold removes: sum over the thresholded coefficients of
    min(|c|, lambda)^2 (the LL band among them only with threshold_ll)."""
    c = make_cube(32, 48, 10, m=3, seed=25)
    lam = 1.3
    o = O.hyres(c["Y"], 3, 10, rank=10, lam=lam, threshold_ll=threshold_ll)
    Rw = (c["Y"].astype(np.float64) - o["X"]) / o["sigma"][:, None, None]
    C = o["C"]
    clipped = np.minimum(np.abs(C), lam) ** 2
    if not threshold_ll:
        clipped[:, : 32 >> 3, : 48 >> 3] = 0.0
    assert abs(np.sum(Rw ** 2) / np.sum(clipped) - 1.0) < 1e-10


def test_selection_tie_break_and_layout():
    S = np.array([[5.0, 3.0, 3.0], [1.0, 1.0, 2.0]])
    S_inf = np.array([4.0, 0.0])
    r, k, T, gap = O.select_rank_lambda(S, S_inf)
    # T[0] = S[0] + S_inf[1] = [5, 3, 3]; T[1] = S[0] + S[1] = [6, 4, 5]
    assert np.array_equal(T, [[5.0, 3.0, 3.0], [6.0, 4.0, 5.0]])
    assert (r, k) == (1, 1) and gap == 0.0


def test_per_component_selection_brute_force():
    """One threshold per kept component: over every rank r and every
    assignment (k_1..k_r) of grid indices, the minimum total SURE
    sum_{i<=r} S_i(k_i) + sum_{i>r} S_i(inf) is the one the selection
    returns, at the rank and indices it returns."""
    import itertools
    rng = np.random.default_rng(7)
    for trial in range(40):
        r_max, K = 3, 4
        S = rng.normal(size=(r_max, K)) * 3.0
        S_inf = rng.normal(size=r_max) * 3.0
        best, arg = np.inf, None
        for r in range(1, r_max + 1):
            for ks in itertools.product(range(K), repeat=r):
                v = sum(S[i, ks[i]] for i in range(r)) + S_inf[r:].sum()
                if v < best:
                    best, arg = v, (r, ks)
        r_star, k, U, gap = O.select_rank_lambda_per_component(S, S_inf)
        assert r_star == arg[0]
        assert tuple(int(x) for x in k[:r_star]) == arg[1]
        assert abs(U[r_star - 1] - best) < 1e-12 and abs(U.min() - best) < 1e-12
        assert gap >= 0.0
        # never above the best shared-threshold total
        assert U.min() <= O.sure_rank_lambda(S, S_inf).min() + 1e-12


def test_per_component_selection_hand_case_and_ties():
    S = np.array([[5.0, 3.0, 3.0], [1.0, 1.0, 2.0]])
    S_inf = np.array([4.0, 0.0])
    r, k, U, gap = O.select_rank_lambda_per_component(S, S_inf)
    # k = [1, 0] (first minimum of each row); U = [3 + 0, 3 + 1]
    assert list(k) == [1, 0] and np.array_equal(U, [3.0, 4.0])
    assert r == 1 and abs(gap - 1.0 / 3.0) < 1e-15
    # equal totals: the smaller rank wins, gap 0
    r, k, U, gap = O.select_rank_lambda_per_component(
        np.array([[2.0, 1.0], [0.0, 0.5]]), np.array([1.0, 0.0]))
    assert np.array_equal(U, [1.0, 1.0]) and r == 1 and gap == 0.0


def test_per_component_reduces_to_shared_when_curves_are_shifts():
    """If every component's SURE curve is one curve plus a constant, all
    components share the minimising index and each rank's per-component
    total is the row minimum of the shared (r, k) table."""
    rng = np.random.default_rng(8)
    f = rng.normal(size=9)
    S = f[None, :] + rng.normal(size=(5, 1)) * 4.0
    S_inf = rng.normal(size=5) * 4.0
    T = O.sure_rank_lambda(S, S_inf)
    r, k, U, _ = O.select_rank_lambda_per_component(S, S_inf)
    r_sh, k_sh, _, _ = O.select_rank_lambda(S, S_inf)
    assert np.allclose(U, T.min(axis=1), rtol=0, atol=1e-12)
    assert r == r_sh and np.all(k == k_sh)


@pytest.mark.parametrize("threshold_ll", [False, True])
def test_sure_levels_sum_to_component_table(threshold_ll):
    """At one threshold for every level the groups add up to the
    component's SURE: n_kept + sum_l S_il(lambda) = S_i(lambda)."""
    rng = np.random.default_rng(9)
    C = rng.normal(size=(3, 24, 40)) * 2.0
    lams = O.lambda_grid(24 * 40, 8)
    S, _ = O.sure_table(C, 3, lams, threshold_ll)
    S_lev = O.sure_table_levels(C, 3, lams, threshold_ll)
    n_kept = 0 if threshold_ll else 3 * 5
    assert np.allclose(n_kept + S_lev.sum(axis=1), S, rtol=0, atol=1e-9)


def test_sure_levels_single_level_image():
    """Only the three level-2 rectangles of a 32 x 48, L = 3 layout (cut
    here by hand) hold nonzero values: the other groups contain zeros only,
    so S_il = N_l - 2 N_l = -3 (H/2^l)(W/2^l); group 2 is the direct
    formula on the hand-cut values."""
    Hp, Wp, L = 32, 48, 3
    rng = np.random.default_rng(10)
    C = np.zeros((1, Hp, Wp))
    h1, w1, h2, w2 = Hp >> 1, Wp >> 1, Hp >> 2, Wp >> 2
    vals = []
    for ys, xs in ((slice(0, h2), slice(w2, w1)), (slice(h2, h1), slice(0, w2)),
                   (slice(h2, h1), slice(w2, w1))):
        block = rng.normal(size=(h2, w2)) * 3.0
        C[0, ys, xs] = block
        vals.append(block.ravel())
    vals = np.abs(np.concatenate(vals))
    lams = np.array([0.0, 0.5, 1.7, 4.0])
    S_lev = O.sure_table_levels(C, L, lams)
    for l in (1, 3):
        assert np.all(S_lev[0, l - 1] == -3.0 * (Hp >> l) * (Wp >> l))
    want = [vals.size - 2.0 * np.sum(vals <= t) + np.sum(np.minimum(vals ** 2, t * t))
            for t in lams]
    assert np.allclose(S_lev[0, 1], want, rtol=0, atol=1e-10)


def test_per_level_selection_brute_force():
    """Over every rank and every assignment of grid indices to the kept
    (component, level) groups, the minimum total SURE is the one the
    per-level selection returns."""
    import itertools
    rng = np.random.default_rng(11)
    for trial in range(25):
        r_max, L, K, n_kept = 2, 2, 3, 5.0
        S_lev = rng.normal(size=(r_max, L, K)) * 3.0
        S_inf = rng.normal(size=r_max) * 6.0
        best, arg = np.inf, None
        for r in range(1, r_max + 1):
            for ks in itertools.product(range(K), repeat=r * L):
                v = sum(n_kept + sum(S_lev[i, l, ks[i * L + l]] for l in range(L))
                        for i in range(r)) + S_inf[r:].sum()
                if v < best:
                    best, arg = v, (r, ks)
        r_star, k, U, gap = O.select_rank_lambda_per_level(S_lev, S_inf, n_kept)
        assert r_star == arg[0]
        assert tuple(int(x) for x in k[:r_star].ravel()) == arg[1]
        assert abs(U.min() - best) < 1e-12 and gap >= 0.0


@pytest.mark.parametrize("threshold_ll", [False, True])
def test_sure_levels_unbiased_monte_carlo(threshold_ll):
    """With a fixed threshold for each (component, level) the sum of the
    group SUREs estimates the whitened squared error without bias (the
    loss thresholds the level rectangles cut by hand)."""
    H, W, p, L, K = 32, 32, 6, 2, 8
    base = make_cube(H, W, p, m=2, seed=13)
    Xw = base["X"].astype(np.float64).reshape(p, -1) / base["sigma"][:, None]
    _, V = O.eig_desc(Xw @ Xw.T)
    lams = O.lambda_grid(H * W, K)
    rng = np.random.default_rng(14)
    kk = rng.integers(0, K, size=(p, L))
    grp = np.ones((H, W), dtype=int)
    grp[: H >> 1, : W >> 1] = 2
    grp[: H >> 2, : W >> 2] = 2 if threshold_ll else 0
    n_kept = 0 if threshold_ll else (H >> 2) * (W >> 2)
    C_clean = O.dwt2((V.T @ Xw).reshape(p, H, W), L)
    diffs = []
    for _ in range(64):
        C = O.dwt2((V.T @ (Xw + rng.standard_normal(Xw.shape))).reshape(p, H, W), L)
        S_lev = O.sure_table_levels(C, L, lams, threshold_ll)
        sure = sum(n_kept + sum(S_lev[i, l, kk[i, l]] for l in range(L)) for i in range(p))
        Ch = C.copy()
        for i in range(p):
            for l in (1, 2):
                m = grp == l
                Ch[i][m] = O.soft_threshold(Ch[i][m], lams[kk[i, l - 1]])
        diffs.append(sure - np.sum((Ch - C_clean) ** 2))
    diffs = np.array(diffs)
    z = diffs.mean() / (diffs.std(ddof=1) / np.sqrt(diffs.size))
    assert abs(z) < 4.0


# ---------------------------------------------------------------- whole path

@pytest.mark.parametrize("threshold_ll", [False, True])
def test_full_rank_residual_per_level_thresholds(threshold_ll):
    """Per-level thresholds at full rank on an unpadded cube: the whitened
    residual energy is sum_{i,l} sum_{group l} min(|c|, lambda_il)^2."""
    c = make_cube(32, 48, 10, m=3, seed=26)
    lam = np.linspace(0.4, 2.2, 10 * 3).reshape(10, 3)
    o = O.hyres(c["Y"], 3, 10, rank=10, lam=lam, lambda_mode="per_level",
                threshold_ll=threshold_ll)
    Rw = (c["Y"].astype(np.float64) - o["X"]) / o["sigma"][:, None, None]
    C = o["C"]
    grp = np.zeros((32, 48), dtype=int)
    for l in (1, 2, 3):
        grp[: 32 >> (l - 1), : 48 >> (l - 1)] = l
    grp[: 32 >> 3, : 48 >> 3] = 3 if threshold_ll else 0
    clipped = 0.0
    for i in range(10):
        for l in (1, 2, 3):
            v = np.abs(C[i][grp == l])
            clipped += np.sum(np.minimum(v, lam[i, l - 1]) ** 2)
    assert abs(np.sum(Rw ** 2) / clipped - 1.0) < 1e-10


def test_per_level_c0_nested_choices():
    """Per-level choices contain the per-component ones, which contain the
    shared one: the minimum SURE can only go down; the planted rank holds."""
    c = make_cube(64, 64, 32, m=4, seed=1)
    o = O.hyres(c["Y"], 2, 8, lambda_mode="per_level")
    oc = O.hyres(c["Y"], 2, 8, lambda_mode="per_component")
    assert o["rank"] == 4
    assert o["U"].min() <= oc["U"].min() + 1e-9 <= o["T"].min() + 2e-9
    assert o["lam_comp"].shape == (4, 2)
    assert O.psnr(c["X"], o["X"]) > O.psnr(c["X"], c["Y"]) + 10.0


def test_per_component_path_is_sum_of_shared_path_increments():
    """Components enter the estimate independently (the DWT, the
    threshold and the back-projection act per component and are linear in
    the kept set), so the per-component estimate is the sum over kept
    components i of [shared path at rank i+1, lambda_{k_i}] minus [shared
    path at rank i, lambda_{k_i}], each run of the shared-threshold path."""
    c = make_cube(48, 40, 16, m=4, seed=24)
    o = O.hyres(c["Y"], 2, 8, lambda_mode="per_component")
    r = o["rank"]
    assert r >= 2 and len(o["lam_comp"]) == r
    assert np.array_equal(o["lam_comp"], o["lams"][o["k_comp"][:r]])
    acc = np.zeros_like(o["X"])
    for i in range(r):
        lam = float(o["lam_comp"][i])
        acc += O.hyres(c["Y"], 2, 8, rank=i + 1, lam=lam)["X"]
        if i > 0:
            acc -= O.hyres(c["Y"], 2, 8, rank=i, lam=lam)["X"]
    assert O.rel_l2(o["X"], acc) < 1e-12
    # the per-component risk estimate is at most the shared one
    assert o["U"].min() <= o["T"].min() + 1e-9 * abs(o["T"].min())


def test_per_component_c0_keeps_planted_rank():
    c = make_cube(64, 64, 32, m=4, seed=1)
    o = O.hyres(c["Y"], 2, 8, lambda_mode="per_component")
    assert o["rank"] == 4
    assert O.psnr(c["X"], o["X"]) > O.psnr(c["X"], c["Y"]) + 10.0


def test_full_rank_zero_lambda_is_identity():
    c = make_cube(30, 45, 10, m=3, seed=21)  # padded to 32 x 48 at L=3
    o = O.hyres(c["Y"], 3, 10, rank=10, lam=0.0)
    assert O.rel_l2(o["X"], c["Y"]) < 1e-12


def test_zero_lambda_is_truncated_whitened_pca():
    c = make_cube(40, 36, 12, m=3, seed=22)
    p, H, W = c["Y"].shape
    o = O.hyres(c["Y"], 2, 12, rank=4, lam=0.0)
    Yw = c["Y"].reshape(p, -1).astype(np.float64).T / o["sigma"]
    U, s, Wt = np.linalg.svd(Yw, full_matrices=False)
    Xw = (U[:, :4] * s[:4]) @ Wt[:4]
    ref = (Xw * o["sigma"]).T.reshape(p, H, W)
    assert O.rel_l2(o["X"], ref) < 1e-10


def test_scale_and_permutation_equivariance():
    c = make_cube(32, 40, 16, m=4, seed=23)
    Y = c["Y"].astype(np.float64)
    o = O.hyres(Y, 2, 8)
    o2 = O.hyres(3.5 * Y, 2, 8)
    assert (o2["rank"], o2["k"]) == (o["rank"], o["k"])
    assert O.rel_l2(o2["X"], 3.5 * o["X"]) < 1e-10
    perm = np.random.default_rng(0).permutation(16)
    o3 = O.hyres(Y[perm], 2, 8)
    assert (o3["rank"], o3["k"]) == (o["rank"], o["k"])
    assert O.rel_l2(o3["X"], o["X"][perm]) < 1e-10


def test_c0_selects_planted_rank_and_denoises():
    c = make_cube(64, 64, 32, m=4, seed=1)
    o = O.hyres(c["Y"], 2, 8)
    assert o["rank"] == 4
    assert O.psnr(c["X"], o["X"]) > O.psnr(c["X"], c["Y"]) + 10.0
    assert O.sam(c["X"], o["X"]) < O.sam(c["X"], c["Y"])


# ---------------------------------------------------------------- gradient form

def _frozen_mask_loss(o, Y_shape, Xc, levels, scale, mask):
    """MSE with the threshold mask frozen: a soft threshold whose kept set is
    fixed is affine in lambda, so the loss is quadratic in the scales."""
    p, H, W = Y_shape
    r = o["rank"]
    C = o["C"][:r]
    lev = o["level_map"]
    Ch = C.copy()
    for i in range(r):
        for l in range(1, levels + 1):
            m = lev == l
            lam = o["lam"] * scale[i, l - 1]
            c = C[i][m]
            Ch[i][m] = np.where(mask[i][m], c - lam * np.sign(c), 0.0)
    Zh = O.idwt2(Ch, levels)[:, :H, :W].reshape(r, H * W)
    Xh = (o["sigma"][:, None] * (o["V"][:, :r] @ Zh)).reshape(p, H, W)
    return O.mse_loss(Xh, Xc)


def test_scaled_forward_at_unit_scale_is_hyres():
    c = make_cube(40, 48, 12, m=3, seed=51)
    o = O.hyres_scaled(c["Y"], 2, 6, np.ones((12, 2)))
    assert O.rel_l2(o["X_scaled"], o["X"]) < 1e-13


def test_whiten_gram_is_gram_of_whitened_cube_and_mse_hand_case():
    """R_w = D^-1 R D^-1 equals the Gram matrix of the cube with each band
    divided by its sigma, formed by a pixel loop (not a matrix product); the
    MSE of a hand case: two voxels off by 1 and 3 among four give 10 / 4."""
    rng = np.random.default_rng(61)
    Y = rng.integers(-4, 5, size=(3, 2, 5)).astype(np.float64)
    sigma = np.array([0.5, 2.0, 4.0])
    Yw = Y / sigma[:, None, None]
    want = np.zeros((3, 3))
    for yy in range(2):
        for xx in range(5):
            v = Yw[:, yy, xx]
            for i in range(3):
                for j in range(3):
                    want[i, j] += v[i] * v[j]
    assert np.allclose(O.whiten_gram(O.gram(Y), sigma), want, rtol=1e-14, atol=0)
    Xh = np.array([[[1.0, 2.0], [3.0, 4.0]]])
    Xc = np.array([[[0.0, 2.0], [3.0, 7.0]]])
    assert O.mse_loss(Xh, Xc) == 10.0 / 4.0


def test_level_map_counts():
    lev = O.level_map(32, 48, 3)
    assert np.count_nonzero(lev == 0) == 4 * 6
    assert np.count_nonzero(lev == 1) == 32 * 48 * 3 // 4
    assert np.count_nonzero(lev == 3) == 3 * 4 * 6


def test_mse_gradient_against_frozen_mask_finite_differences():
    """With the kept set frozen the loss is exactly quadratic in s, so central
    differences (h = 1e-3) equal the analytic adjoint to rounding."""
    c = make_cube(48, 40, 16, m=3, seed=41)
    levels, r_max = 2, 8
    rng = np.random.default_rng(0)
    s = 1.0 + 0.2 * rng.standard_normal((16, levels))
    o = O.hyres_scaled(c["Y"], levels, r_max, s)
    G = 2.0 * (o["X_scaled"] - c["X"]) / c["X"].size
    g, _ = O.hyres_scaled_grad(c["Y"], G, levels, r_max, s)
    r = o["rank"]
    mask = np.zeros(o["C"][:r].shape, dtype=bool)
    for i in range(r):
        for l in range(1, levels + 1):
            m = o["level_map"] == l
            mask[i][m] = np.abs(o["C"][i][m]) > o["lam"] * s[i, l - 1]
    h = 1e-3
    fd = np.zeros_like(s)
    for i in range(r):
        for l in range(levels):
            e = np.zeros_like(s)
            e[i, l] = h
            fd[i, l] = (_frozen_mask_loss(o, c["Y"].shape, c["X"], levels, s + e, mask)
                        - _frozen_mask_loss(o, c["Y"].shape, c["X"], levels, s - e, mask)) / (2 * h)
    assert np.max(np.abs(fd[:r] - g[:r])) < 1e-7 * max(1.0, np.max(np.abs(g[:r])))
    assert np.all(g[r:] == 0.0)
    # mask free: the kinks move only a few coefficients, so raw differences
    # still agree to about 1 %
    raw = np.zeros_like(s)
    for i in range(r):
        for l in range(levels):
            e = np.zeros_like(s)
            e[i, l] = h
            raw[i, l] = (O.mse_loss(O.hyres_scaled(c["Y"], levels, r_max, s + e)["X_scaled"], c["X"])
                         - O.mse_loss(O.hyres_scaled(c["Y"], levels, r_max, s - e)["X_scaled"], c["X"])) / (2 * h)
    assert np.linalg.norm(raw[:r] - g[:r]) <= 1e-2 * np.linalg.norm(g[:r])


def test_sure_loss_gradient_continuous_part():
    """The SURE loss is piecewise smooth in s: its count term jumps, the rest
    is sum min(c^2, lam^2). Central differences of that continuous part match
    the stated gradient 2 lam* lam #{|c| > lam}."""
    c = make_cube(48, 40, 16, m=3, seed=42)
    levels, r_max = 2, 8
    s = np.full((16, levels), 1.1)
    o = O.hyres_scaled(c["Y"], levels, r_max, s)
    val, g = O.sure_loss_scaled(o, levels, s)
    r = o["rank"]
    h = 1e-4
    for i in range(r):
        for l in range(levels):
            m = o["level_map"] == l + 1
            cc = np.abs(o["C"][i][m])

            def cont(si):
                lam = o["lam"] * si
                return np.sum(np.minimum(cc * cc, lam * lam))
            fd = (cont(s[i, l] + h) - cont(s[i, l] - h)) / (2 * h)
            assert abs(fd - g[i, l]) <= 1e-6 * max(1.0, abs(g[i, l]))
    # at s = 1 the per-level SURE equals the selection table's entry for (r*, k*)
    o1 = O.hyres_scaled(c["Y"], levels, r_max, np.ones((16, levels)))
    v1, _ = O.sure_loss_scaled(o1, levels, np.ones((16, levels)))
    assert abs(v1 - np.sum(o1["S"][: o1["rank"], o1["k"]])) < 1e-6 * abs(v1)


# ---------------------------------------------------------------- HySime

def test_hysime_correlations_closed_form_from_inverse_gram():
    """The regression residual of band b is Y q_b / q_bb (q_b the b-th column
    of Q = (Y^T Y)^-1), so with R = Y^T Y and D_Q = diag(Q):
    R_n = D_Q^-1 Q D_Q^-1 / n, Y^T W = D_Q^-1 and
    R_x = (R - 2 D_Q^-1 + D_Q^-1 Q D_Q^-1) / n: a route through the Gram
    matrix alone, against the oracle's per-band least squares on the data."""
    c = make_cube(40, 36, 12, m=3, seed=27)
    h = O.hysime(c["Y"])
    Yf = c["Y"].reshape(12, -1).astype(np.float64).T
    n = Yf.shape[0]
    R = Yf.T @ Yf
    Q = np.linalg.inv(R)
    Di = np.diag(1.0 / np.diag(Q))
    Rn = Di @ Q @ Di / n
    Rx = (R - 2.0 * Di + Di @ Q @ Di) / n
    assert np.allclose(h["Ry"], R / n, rtol=1e-12, atol=0)
    assert np.max(np.abs(h["Rn"] - Rn)) < 1e-9 * np.max(np.abs(Rn))
    assert np.max(np.abs(h["Rx"] - Rx)) < 1e-9 * np.max(np.abs(Rx))


def test_hysime_selection_minimises_subspace_error_brute_force():
    """Over every subset S of the eigenvectors, the projection error
    tr((I - P_S) R_y) + 2 tr(P_S R_n) (P_S the projector on S) is smallest
    for the set HySime keeps, {i : delta_i < 0}."""
    import itertools
    rng = np.random.default_rng(15)
    for trial in range(20):
        p = 6
        A = rng.normal(size=(p, p))
        Ry = A @ A.T + 0.1 * np.eye(p)
        B = rng.normal(size=(p, p)) * 0.5
        Rn = B @ B.T + 0.05 * np.eye(p)
        _, E = np.linalg.eigh(rng.normal(size=(p, p)) + rng.normal(size=(p, p)).T)
        k, idx, delta = O.hysime_select(E, Ry, Rn)
        best, arg = np.inf, None
        for size in range(p + 1):
            for S in itertools.combinations(range(p), size):
                P = E[:, list(S)] @ E[:, list(S)].T
                cost = np.trace((np.eye(p) - P) @ Ry) + 2.0 * np.trace(P @ Rn)
                if cost < best - 1e-12:
                    best, arg = cost, set(S)
        assert set(int(i) for i in idx) == arg and k == len(arg)
        assert np.all(np.diff(delta[idx]) >= 0)


@pytest.mark.parametrize("m,snr", [(3, 30.0), (5, 30.0), (4, 10.0)])
def test_hysime_recovers_planted_dimension(m, snr):
    c = make_cube(64, 64, 32, m=m, snr_db=snr, seed=7)
    h = O.hysime(c["Y"])
    assert h["k"] == m
    # the subspace holds the clean cube: its projection keeps > 99.9 % of it
    Xf = c["X"].reshape(32, -1).astype(np.float64)
    P = h["E"] @ h["E"].T
    assert np.linalg.norm(P @ Xf) / np.linalg.norm(Xf) > 0.999


def test_hysime_white_noise_has_no_signal_subspace():
    Z = np.random.default_rng(16).standard_normal((16, 64, 64)).astype(np.float32)
    assert O.hysime(Z)["k"] == 0


def test_hysime_scale_and_band_permutation():
    c = make_cube(48, 48, 20, m=4, snr_db=25.0, seed=28)
    Y = c["Y"].astype(np.float64)
    h = O.hysime(Y)
    h2 = O.hysime(2.5 * Y)
    assert h2["k"] == h["k"] and np.allclose(np.abs(h2["E"]), np.abs(h["E"]), atol=1e-8)
    perm = np.random.default_rng(1).permutation(20)
    h3 = O.hysime(Y[perm])
    assert h3["k"] == h["k"]
    P, P3 = h["E"] @ h["E"].T, h3["E"] @ h3["E"].T
    assert np.allclose(P3, P[np.ix_(perm, perm)], atol=1e-8)


# ---------------------------------------------------------------- lambda grid

def test_lambda_grid_golden_values():
    """Grid points against decimal values worked out at 40 digits
    (tests/golden/lambda_grid.txt): N = 675,840 is the padded pixel count of
    the 349 x 1905 cube at five levels (352 x 1920), N = 4096 the 64 x 64
    cube's. A log10 in place of ln, a missing factor 2 or a K in place of
    K - 1 each miss these by far more than the tolerance."""
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", "lambda_grid.txt")
    rows = [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]
    assert len(rows) == 5
    for N, K, k, val in rows:
        lams = O.lambda_grid(int(N), int(K))
        assert lams.shape == (int(K),)
        assert abs(lams[int(k)] - float(val)) < 4e-15 * float(val)


def test_lambda_grid_top_is_universal_threshold():
    """The top point lambda_max satisfies N exp(-lambda_max^2 / 2) = 1, the
    defining property of the universal threshold (N times the Gaussian tail
    density ratio at lambda_max is one); lambda_0 = 0 and the grid is
    uniform."""
    for N in (2, 17, 4096, 675840, 10 ** 9):
        lams = O.lambda_grid(N, 64)
        assert lams[0] == 0.0
        assert abs(N * np.exp(-lams[-1] ** 2 / 2.0) - 1.0) < 1e-12
        d = np.diff(lams)
        assert np.max(np.abs(d - d[0])) < 1e-14 * lams[-1]
    assert O.lambda_grid(4096, 2).tolist() == [0.0, O.lambda_grid(4096, 64)[-1]]


# ---------------------------------------------------------------- metrics

def test_rel_l2_hand_case_and_operand_order():
    """||est - ref|| / ||ref||: ref = (3, 4) has norm 5; est = (3, 5.25)
    differs by 1.25 -> 0.25. With est = (6, 8) the error norm is 5 -> 1.0,
    and the swapped call divides by ||(6, 8)|| = 10 -> 0.5, so the
    denominator is the second argument."""
    ref = np.array([[3.0, 4.0]])
    assert abs(O.rel_l2(np.array([[3.0, 5.25]]), ref) - 0.25) < 1e-15
    assert abs(O.rel_l2(np.array([[6.0, 8.0]]), ref) - 1.0) < 1e-15
    assert abs(O.rel_l2(ref, np.array([[6.0, 8.0]])) - 0.5) < 1e-15
    assert O.rel_l2(ref, ref) == 0.0


def test_psnr_hand_case():
    """Two bands of two pixels. Band 0: clean (1, 2), estimate (1, 1): MSE
    1/2, peak 2 -> 10 log10(4 / 0.5) = 30 log10 2. Band 1: clean (3, 4),
    estimate (3, 5): MSE 1/2, peak 4 -> 10 log10(16 / 0.5) = 50 log10 2.
    Mean over bands 40 log10 2 = 12.0412 dB. The peak comes from the clean
    band: taking it from the estimate (1 and 5) gives another value, and so
    does one MSE over the whole cube."""
    clean = np.array([[1.0, 2.0], [3.0, 4.0]])
    est = np.array([[1.0, 1.0], [3.0, 5.0]])
    log2 = 0.30102999566398119521373889472449302676818988146211   # log10(2)
    assert abs(O.psnr(clean, est) - 40.0 * log2) < 1e-13
    # three-axis input [p][H][W] reads the same
    assert abs(O.psnr(clean.reshape(2, 1, 2), est.reshape(2, 1, 2)) - 40.0 * log2) < 1e-13


def test_sam_hand_case():
    """Pixel 0: clean (1, 0), estimate (1, 1) -> angle pi/4. Pixel 1: clean
    (0, 1), estimate (0, 2) -> angle 0 (scale does not matter). Mean pi/8.
    The layout is [band][pixel]: the transposed reading pairs (1, 0) with
    (1, 0) and (0, 1) with (1, 2) and gives a different mean."""
    clean = np.array([[1.0, 0.0], [0.0, 1.0]])
    est = np.array([[1.0, 0.0], [1.0, 2.0]])
    assert abs(O.sam(clean, est) - np.pi / 8.0) < 1e-15
    assert abs(O.sam(clean.T, est.T) - np.pi / 8.0) > 1e-3
    assert O.sam(clean, 3.0 * clean) == 0.0


# ---------------------------------------------------------------- HyMiNoR

def _tvl1_lp(h, lam):
    """Exact minimum of ||h - x||_1 + lam (||Dx x||_1 + ||Dy x||_1) for one
    small periodic image, as a linear program (scipy's HiGHS): variables x,
    e >= |h - x|, f >= |Dx x|, g >= |Dy x|."""
    from scipy.optimize import linprog
    H, W = h.shape
    n = H * W
    idx = np.arange(n).reshape(H, W)
    right = np.roll(idx, -1, axis=1).ravel()
    down = np.roll(idx, -1, axis=0).ravel()
    nv = 4 * n
    c = np.concatenate([np.zeros(n), np.ones(n), lam * np.ones(n), lam * np.ones(n)])
    rows, rhs = [], []
    hv = h.ravel()
    for k in range(n):
        for sgn in (1.0, -1.0):
            r = np.zeros(nv); r[k] = -sgn; r[n + k] = -1.0; rows.append(r); rhs.append(-sgn * hv[k])
            r = np.zeros(nv); r[right[k]] += sgn; r[k] -= sgn; r[2 * n + k] = -1.0
            rows.append(r); rhs.append(0.0)
            r = np.zeros(nv); r[down[k]] += sgn; r[k] -= sgn; r[3 * n + k] = -1.0
            rows.append(r); rhs.append(0.0)
    bounds = [(None, None)] * n + [(0, None)] * (3 * n)
    res = linprog(c, A_ub=np.array(rows), b_ub=np.array(rhs), bounds=bounds, method="highs")
    assert res.status == 0
    return res.fun


def test_periodic_differences_hand_case():
    x = np.array([[1.0, 2.0, 4.0], [7.0, 11.0, 16.0]])
    import importlib
    HM = importlib.import_module("oracle.hyminor")
    assert HM.dx(x).tolist() == [[1.0, 2.0, -3.0], [4.0, 5.0, -9.0]]
    assert HM.dy(x).tolist() == [[6.0, 9.0, 12.0], [-6.0, -9.0, -12.0]]
    # the transposes satisfy <Dx x, z> = <x, Dx^T z>
    z = np.arange(6.0).reshape(2, 3) - 2.5
    assert abs(np.sum(HM.dx(x) * z) - np.sum(x * HM.dxT(z))) < 1e-12
    assert abs(np.sum(HM.dy(x) * z) - np.sum(x * HM.dyT(z))) < 1e-12


@pytest.mark.parametrize("lam", [0.15, 0.5, 1.0])
def test_tvl1_split_bregman_reaches_the_lp_optimum(lam):
    """The split-Bregman iteration (two Jacobi sweeps per step) run long
    enough reaches the minimum that a linear program (an independent route:
    HiGHS) finds for the same l1-l1 objective, on small periodic images with
    outliers."""
    rng = np.random.default_rng(7)
    for trial in range(3):
        h = np.cumsum(rng.standard_normal((5, 6)) * 0.3, axis=1)
        h[rng.integers(0, 5), rng.integers(0, 6)] += 3.0     # one outlier
        x = O.tvl1_split_bregman(h, lam=lam, mu=10.0, iters=6000)
        f_lp = _tvl1_lp(h, lam)
        f_sb = O.tvl1_objective(h, x, lam)
        assert f_sb <= f_lp + 1e-5 * (1.0 + f_lp), (trial, f_sb, f_lp)


def test_tvl1_removes_an_isolated_spike():
    """A piecewise-constant image with one spike of height 2 at an interior
    pixel of a flat region: keeping it costs 4 lam * 2 in the penalty,
    removing it 2 in the data term, so at lam = 1 the minimiser is the image
    without the spike (matched exactly by the data term)."""
    clean = np.ones((8, 8))
    clean[:, 5:] = 3.0
    h = clean.copy()
    h[3, 2] += 2.0
    x = O.tvl1_split_bregman(h, lam=1.0, mu=10.0, iters=4000)
    assert np.max(np.abs(x - clean)) < 1e-5, np.max(np.abs(x - clean))


def test_tvl1_zero_penalty_is_identity():
    """lam = 0 leaves only ||h - x||_1, minimised by x = h."""
    rng = np.random.default_rng(3)
    h = rng.standard_normal((2, 6, 7))
    x = O.tvl1_split_bregman(h, lam=0.0, mu=10.0, iters=3000)
    assert np.max(np.abs(x - h)) < 1e-6


def test_hyminor_scale_equivariant_and_cleans_sparse_noise():
    """HyMiNoR(a Y) = a HyMiNoR(Y) (the stage is normalised by max |HyRes(Y)|),
    and on cubes with Gaussian plus salt-and-pepper or stripe noise the
    l1-l1 stage brings the estimate closer to the clean cube than HyRes
    alone."""
    from synth import noise as N
    c = make_cube(48, 48, 24, m=3, seed=11)
    Yn, _ = N.salt_and_pepper(c["Y"], 0.02, seed=2)
    o = O.hyminor(Yn, 2, 6)
    o2 = O.hyminor(Yn * np.float32(4.0), 2, 6)
    assert O.rel_l2(o2["X"], 4.0 * o["X"]) < 1e-6
    assert O.rel_l2(o["X"], c["X"]) < 0.9 * O.rel_l2(o["G"], c["X"])
    Ys, _ = N.stripes(c["Y"], 8, band_fraction=0.3, amplitude=1.0, seed=2)
    o3 = O.hyminor(Ys, 2, 6)
    assert O.rel_l2(o3["X"], c["X"]) < 0.9 * O.rel_l2(o3["G"], c["X"])


# ---------------------------------------------------------------- Gram matrix

def test_gram_hand_case_and_brute_force():
    """R = Y^T Y with pixels as rows and bands as columns, input [band][H][W].
    Hand case: bands (1, 2, 3) and (4, 5, 6) over three pixels give
    R = [[14, 32], [32, 77]]. A transposed reading (pixels as columns) would
    give a 3 x 3 matrix. Brute force: a triple loop over bands and pixels on
    a small random cube, exact in float64 for small integer entries."""
    Y = np.array([[[1.0, 2.0, 3.0]], [[4.0, 5.0, 6.0]]], dtype=np.float32)   # p=2, H=1, W=3
    assert O.gram(Y).tolist() == [[14.0, 32.0], [32.0, 77.0]]
    rng = np.random.default_rng(5)
    Y = rng.integers(-8, 9, size=(5, 3, 4)).astype(np.float32)
    R = O.gram(Y)
    p = Y.shape[0]
    for a in range(p):
        for b in range(p):
            s = 0.0
            for y in range(3):
                for x in range(4):
                    s += float(Y[a, y, x]) * float(Y[b, y, x])
            assert R[a, b] == s


# ---------------------------------------------------------------- FORPDN

def _forpdn():
    import importlib
    return importlib.import_module("oracle.forpdn")


def test_forpdn_smoother_two_bands_hand_case():
    """p = 2: D^T D = [[1, -1], [-1, 1]], so (I + lam D^T D)^-1 =
    [[1 + lam, lam], [lam, 1 + lam]] / (1 + 2 lam)."""
    F = _forpdn()
    for lam in (0.0, 0.25, 3.0):
        S = F.smoother(2, lam)
        ref = np.array([[1 + lam, lam], [lam, 1 + lam]]) / (1 + 2 * lam)
        assert np.max(np.abs(S - ref)) < 1e-15
    D = F.diff_operator(4)
    assert D.tolist() == [[-1, 1, 0, 0], [0, -1, 1, 0], [0, 0, -1, 1]]


def test_forpdn_smoother_limits():
    """lam = 0 is the identity; lam -> infinity projects every spectrum onto
    the constants (the null space of D), 1 1^T / p."""
    F = _forpdn()
    for p in (3, 7, 32):
        assert np.max(np.abs(F.smoother(p, 0.0) - np.eye(p))) < 1e-15
        assert np.max(np.abs(F.smoother(p, 1e9) - np.ones((p, p)) / p)) < 1e-5


def test_forpdn_lambda_grid():
    F = _forpdn()
    lams = F.forpdn_lambda_grid(64)
    assert lams[0] == 0.0 and abs(lams[1] - 1e-3) < 1e-18 and abs(lams[-1] - 1e4) < 1e-9
    r = lams[2:] / lams[1:-1]
    assert np.max(np.abs(r - r[0])) < 1e-12 * r[0]


def test_forpdn_sure_is_unbiased_monte_carlo():
    """E[SURE(lam)] = E ||C S - X||^2 for C = X + noise with independent
    band variances sigma_b^2: over 400 draws the mean SURE and the mean true
    error agree within 4 standard errors for several lam."""
    F = _forpdn()
    rng = np.random.default_rng(12)
    p, N = 12, 300
    X = np.cumsum(rng.standard_normal((N, p)) * 0.4, axis=1)        # smooth-ish spectra
    sigma = rng.uniform(0.5, 2.0, p)
    for lam in (0.1, 1.0, 10.0):
        S = F.smoother(p, lam)
        sures, errs = [], []
        for _ in range(400):
            C = X + rng.standard_normal((N, p)) * sigma
            sures.append(F.sure_group(C.T @ C, N, sigma ** 2, lam))
            errs.append(float(np.sum((C @ S - X) ** 2)))
        d = np.array(sures) - np.array(errs)
        se = np.std(d) / np.sqrt(len(d))
        assert abs(np.mean(d)) < 4 * se + 1e-9, (lam, np.mean(d), se)


def test_forpdn_denoises_and_respects_symmetries():
    """Scale equivariance (FORPDN(4 Y) = 4 FORPDN(Y), the same grid indices;
    a power of two keeps the float32 input exact);
    reversing the band order commutes with the estimate (D^T D and the SURE
    are invariant under it); zero smoothing of every group reproduces Y; and
    on the 64 x 64 x 32 cube the estimate beats the noisy input by more than
    6 dB."""
    F = _forpdn()
    c = make_cube(64, 64, 32, m=4, seed=1)
    Y = c["Y"]
    o = F.forpdn(Y, 2)
    o2 = F.forpdn(Y * np.float32(4.0), 2)
    assert o2["k"].tolist() == o["k"].tolist()
    assert O.rel_l2(o2["X"], 4.0 * o["X"]) < 1e-12
    o3 = F.forpdn(Y[::-1].copy(), 2)
    assert o3["k"].tolist() == o["k"].tolist()
    assert O.rel_l2(o3["X"][::-1], o["X"]) < 1e-10
    assert O.psnr(c["X"], o["X"]) > O.psnr(c["X"], Y) + 6.0
    # group sizes cover the padded image once
    lev = O.level_map(64, 64, 2)
    assert sum(int(np.sum(lev == g)) for g in range(3)) == 64 * 64


# ---------------------------------------------------------------- WSRRR

def _wsrrr():
    import importlib
    return importlib.import_module("oracle.wsrrr")


def test_wsrrr_zero_iterations_is_hyres_and_objective_decreases():
    """No V-step leaves HyRes's estimate; each half-step is an exact block
    minimisation, so the objective never increases (C0 and a cube with
    padded sides)."""
    Wm = _wsrrr()
    for (H, W, p, m, seed, L, r) in [(64, 64, 32, 4, 1, 2, 8), (50, 45, 24, 3, 9, 3, 6)]:
        c = make_cube(H, W, p, m=m, seed=seed)
        g = O.hyres(c["Y"], L, r)
        o0 = Wm.wsrrr(c["Y"], L, r, iters=0, hy=g)
        assert O.rel_l2(o0["X"], g["X"]) < 1e-12
        o = Wm.wsrrr(c["Y"], L, r, iters=6, hy=g)
        d = np.diff(o["J"])
        assert np.all(d <= 1e-12 * abs(o["J"][0])), d
        assert o["J"][-1] < o["J"][0]


def test_wsrrr_without_threshold_keeps_the_eigenvectors():
    """lam = 0 on an unpadded cube: B = W2^T Yw V, so Yw^T W2 B = (Yw^T Yw) V
    = V Lambda for eigenvectors V, whose polar factor is V itself."""
    Wm = _wsrrr()
    c = make_cube(64, 64, 32, m=4, seed=1)
    g = O.hyres(c["Y"], 2, 8, rank=5, lam=0.0)
    o = Wm.wsrrr(c["Y"], 2, 8, iters=3, hy=g)
    assert np.max(np.abs(o["V"] - g["V"][:, :5])) < 1e-10


def test_wsrrr_polar_factor_solves_procrustes():
    """polar(M) maximises tr(V^T M) over matrices with orthonormal columns:
    the maximum is the sum of M's singular values, and no random orthonormal
    V exceeds it."""
    Wm = _wsrrr()
    rng = np.random.default_rng(4)
    M = rng.standard_normal((12, 4)) @ np.diag([5.0, 2.0, 1.0, 0.1])
    P = Wm.polar(M)
    assert np.max(np.abs(P.T @ P - np.eye(4))) < 1e-13
    best = np.trace(P.T @ M)
    assert abs(best - np.sum(np.linalg.svd(M, compute_uv=False))) < 1e-12
    for _ in range(200):
        Qr, _ = np.linalg.qr(rng.standard_normal((12, 4)))
        assert np.trace(Qr.T @ M) <= best + 1e-12


def test_wsrrr_scale_equivariant():
    Wm = _wsrrr()
    c = make_cube(48, 48, 16, m=3, seed=6)
    o = Wm.wsrrr(c["Y"], 2, 6, iters=3)
    o4 = Wm.wsrrr(c["Y"] * np.float32(4.0), 2, 6, iters=3)
    assert o4["rank"] == o["rank"]
    assert O.rel_l2(o4["X"], 4.0 * o["X"]) < 1e-10
