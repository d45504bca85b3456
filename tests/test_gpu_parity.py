"""GPU parity: every C-ABI stage of the CUDA path against the FP64 oracle on
the same seeded float32 inputs.

Tolerances: the whole path must match the oracle to relative L2 <= 1e-5 with
the identical (rank, lambda) choice; single stages are held to tolerances
derived from float32 arithmetic on the stage (stated per test).
"""

import numpy as np
import pytest
import torch

import oracle as O
from selection_checks import check_per_level_choice
from synth import make_cube

pytestmark = pytest.mark.gpu

REL_L2_PATH = 1e-5


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# ------------------------------------------------------------------- DWT

@pytest.mark.parametrize("B,H,W,L", [
    (1, 64, 64, 2),      # C0 image size, one tile row
    (3, 100, 150, 3),    # ragged: padded to 104 x 152, several tiles
    (2, 349, 1905, 5),   # C1 component size
    (1, 5, 7, 2),        # tiny: tiles larger than the image, wrap inside a tile
    (4, 33, 65, 1),      # single level, odd sides
    (2, 128, 256, 4),    # levels 2-4 fused in one block per image (both shared buffers)
])
def test_dwt2_matches_oracle(hyde, B, H, W, L):
    rng = np.random.default_rng(B * 1000 + H + W)
    x = rng.standard_normal((B, H, W)).astype(np.float32) * 4 + 1
    Hp, Wp = O.padded_shape(H, W, L)
    ref = O.dwt2(O.pad_symmetric(x.astype(np.float64), Hp, Wp), L)
    got = hyde.dwt2(_t(x), L).cpu().numpy().astype(np.float64)
    # orthogonal transform: float32 rounding of ~4 taps x 2 passes per level
    assert got.shape == ref.shape
    assert O.rel_l2(got, ref) < 2e-7 * (L + 1)
    assert np.max(np.abs(got - ref)) < 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("B,H,W,L", [(2, 64, 64, 2), (3, 100, 150, 3), (1, 349, 1905, 5),
                                     (2, 128, 256, 4), (1, 120, 250, 4)])
def test_idwt2_matches_oracle_and_inverts(hyde, B, H, W, L):
    rng = np.random.default_rng(7 + H)
    Hp, Wp = O.padded_shape(H, W, L)
    c = rng.standard_normal((B, Hp, Wp)).astype(np.float32)
    ref = O.idwt2(c.astype(np.float64), L)[:, :H, :W]
    got = hyde.idwt2(_t(c), H, W, L).cpu().numpy()
    assert O.rel_l2(got, ref) < 2e-7 * (L + 1)
    x = rng.standard_normal((B, H, W)).astype(np.float32)
    back = hyde.idwt2(hyde.dwt2(_t(x), L), H, W, L).cpu().numpy()
    assert O.rel_l2(back, x) < 1e-6


# ------------------------------------------------------------------ Gram

@pytest.mark.parametrize("p,H,W", [(32, 64, 64), (37, 33, 51), (144, 97, 131), (8, 1, 1000),
                                   (200, 40, 41), (3, 17, 3)])
def test_gram_matches_oracle(hyde, p, H, W):
    rng = np.random.default_rng(p + H)
    Y = (rng.standard_normal((p, H, W)) + 0.5).astype(np.float32)
    ref = O.gram(Y)
    got = hyde.gram(_t(Y)).cpu().numpy()
    assert np.allclose(got, got.T)
    # float32 partial sums over <= a few thousand pixels, combined in double
    assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(ref))


def test_gram_full_c1(hyde):
    c = make_cube(349, 1905, 144, m=12, seed=2)
    ref = O.gram(c["Y"])
    got = hyde.gram(_t(c["Y"])).cpu().numpy()
    assert np.max(np.abs(got - ref) / np.sqrt(np.outer(np.diag(ref), np.diag(ref)))) < 2e-6


# ------------------------------------------------------------ noise level

@pytest.mark.parametrize("H,W,p,m,seed", [
    (64, 64, 32, 4, 1), (128, 128, 64, 8, 5), (45, 70, 24, 3, 9),
    (60, 64, 150, 5, 11),    # 16 x 16 threads, 10 x 10 register tiles
    (60, 66, 176, 5, 12),    # 16 x 16 threads, 11 x 11 tiles
    (64, 72, 200, 6, 13),    # 13 x 13 tiles at p = 200 (the sliding-window scenes)
    (64, 80, 230, 6, 14),    # shared-memory kernel
])
def test_noise_est_matches_oracle(hyde, H, W, p, m, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    ref = O.noise_est_regression(O.gram(c["Y"]), H * W)
    sigma, status = hyde.noise_est(_t(c["Y"]))
    assert int(status.item()) == 0
    # float Gram partials (~1e-7) through a Schur complement of condition
    # ~1e3, one double Newton step on the float inverse's diagonal
    assert np.max(np.abs(sigma.cpu().numpy() / ref - 1)) < 2e-5


def test_noise_est_duplicate_band_reports_numeric(hyde):
    c = make_cube(32, 32, 8, m=2, seed=3)
    Y = c["Y"].copy()
    Y[5] = Y[2]          # exactly collinear bands: R is singular
    _, status = hyde.noise_est(_t(Y))
    assert int(status.item()) == 3


# -------------------------------------------------------------------- eig

@pytest.mark.parametrize("cfg", ["c0", "c4"])
def test_eig_matches_oracle(hyde, cfg):
    shapes = {"c0": (64, 64, 32, 4, 1, 8), "c4": (128, 128, 64, 8, 5, 16)}
    H, W, p, m, seed, r = shapes[cfg]
    c = make_cube(H, W, p, m=m, seed=seed)
    R = O.gram(c["Y"])
    Rw = O.whiten_gram(R, O.noise_est_regression(R, H * W))
    e_ref, V_ref = O.eig_desc(Rw)
    evals, V, status = hyde.eig_sym_top(_t(Rw), r)
    assert int(status.item()) == 0
    evals = evals.cpu().numpy()
    V = V.cpu().numpy()
    # eigenvalues: float32 accuracy relative to the largest one
    assert np.max(np.abs(evals - e_ref[:r])) < 5e-6 * e_ref[0]
    assert np.max(np.abs(V.T @ V - np.eye(r))) < 1e-5
    # well-separated eigenvectors individually; the whole r-space as a projector
    gaps = np.abs(np.diff(e_ref[: r + 1])) / e_ref[0]
    for i in range(r):
        gap = min(gaps[i], gaps[i - 1] if i > 0 else np.inf)
        if gap > 1e-3:
            assert abs(V[:, i] @ V_ref[:, i]) > 1 - 1e-6
    # residual ||Rw v - e v|| relative to ||Rw||
    res = np.linalg.norm(Rw @ V - V * evals, axis=0) / e_ref[0]
    assert np.max(res) < 1e-5


@pytest.mark.parametrize("H,W,p,m,seed,r", [
    (349, 1905, 144, 12, 2, 20),    # the benchmark cube's whitened Gram matrix
    (88, 48, 200, 12, 4, 20),       # a small sliding window: n ~ 21 p
    (128, 128, 200, 12, 6, 20),     # a large sliding window
])
def test_eig_at_size(hyde, H, W, p, m, seed, r):
    """The eigensolver on the whitened Gram matrices it meets on the
    benchmark cube (p = 144) and on sliding windows (p = 200), fed the
    oracle's FP64 matrix. Bounds of a float32 solver, with u = 2^-24 and e_0
    the largest eigenvalue: eigenvalues and residuals ||A v - e v|| within
    p u e_0; an eigenvector within sin(angle) <= 2 p u / g + 1e-6 of the
    oracle's, g its gap to the neighbouring eigenvalues relative to e_0; the
    leading invariant subspace up to the largest relative gap g* inside the
    top r (signal against noise) within 2 p u / g* as a projector. (LAPACK's
    float32 solver meets each bound with a factor of 10 or more to spare on
    these three matrices.)"""
    c = make_cube(H, W, p, m=m, seed=seed)
    R = O.gram(c["Y"])
    Rw = O.whiten_gram(R, O.noise_est_regression(R, H * W))
    e_ref, V_ref = O.eig_desc(Rw)
    evals, V, status = hyde.eig_sym_top(_t(Rw), r)
    assert int(status.item()) == 0
    evals = evals.cpu().numpy()
    V = V.cpu().numpy()
    e0, pu = e_ref[0], p * 2.0 ** -24
    assert np.max(np.abs(evals - e_ref[:r])) < pu * e0, np.max(np.abs(evals - e_ref[:r])) / e0
    assert np.max(np.abs(V.T @ V - np.eye(r))) < 1e-5
    res = np.linalg.norm(Rw @ V - V * evals, axis=0) / e0
    assert np.max(res) < pu, np.max(res)
    g = np.abs(np.diff(e_ref[: r + 1])) / e0
    for i in range(r):
        gap = min(g[i], g[i - 1] if i > 0 else np.inf)
        assert _sin_angle(V[:, i], V_ref[:, i]) <= 2 * pu / gap + 1e-6, (i, gap)
    s = int(np.argmax(g[: r - 1])) + 1          # leading block 0..s-1
    P = V[:, :s] @ V[:, :s].T
    Pr = V_ref[:, :s] @ V_ref[:, :s].T
    assert np.linalg.norm(P - Pr, 2) <= 2 * pu / g[s - 1], (s, g[s - 1])
    # the sign rule: the entry of largest magnitude is positive
    piv = np.argmax(np.abs(V), axis=0)
    assert np.all(V[piv, np.arange(r)] > 0)


def _sin_angle(v, w):
    """Sine of the angle between the lines through v and w."""
    v = v / np.linalg.norm(v)
    w = w / np.linalg.norm(w)
    return float(np.linalg.norm(v - (v @ w) * w))


# ------------------------------------------------------------------- SURE

def test_sure_table_matches_oracle(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    o = O.hyres(c["Y"], 2, 8)
    C32 = o["C"].astype(np.float32)
    S_ref, Sinf_ref = O.sure_table(C32.astype(np.float64), 2, o["lams"])
    S, S_inf = hyde.sure_table(_t(C32), 2, 64)
    S = S.cpu().numpy()
    # counts are exact integers; a coefficient within rounding of a grid point
    # may land on either side (changes S by at most 2 + lambda^2 - c^2 ~ 2)
    assert np.max(np.abs(S - S_ref)) < 4.0 + 1e-6 * np.max(np.abs(S_ref))
    assert np.max(np.abs(S_inf.cpu().numpy() - Sinf_ref)) < 1e-6 * np.max(np.abs(Sinf_ref)) + 1e-3


# ------------------------------------------------------------ whole path

def _check_hyres(hyde, Y, L, r_max, K=64, tol=REL_L2_PATH, threshold_ll=False):
    o = O.hyres(Y, L, r_max, K, threshold_ll=threshold_ll)
    p, H, W = Y.shape
    h = hyde.HyRes(p, H, W, L, r_max, K, threshold_ll=threshold_ll)
    X = h(_t(Y)).cpu().numpy()
    info = h.result_info()
    mid = h.intermediates()
    assert info["status"] == 0
    assert (info["rank"], info["lambda_index"]) == (o["rank"], o["k"]), (info, o["rank"], o["k"], o["gap"])
    assert np.max(np.abs(mid["sigma"].cpu().numpy() / o["sigma"] - 1)) < 2e-5
    err = O.rel_l2(X, o["X"])
    assert err < tol, err
    _check_per_band(X, o["X"], 10 * tol)
    return o, X, info, mid


def _check_per_band(X, ref, tol):
    """Per-band relative L2 error and per-band largest absolute error
    (relative to the band's largest magnitude), so that a defect confined to
    a few rows or columns of some bands (the cropped padding at the bottom
    and right edges, one band's weights) cannot hide inside the whole-cube
    norm."""
    p = ref.shape[0]
    d = (np.asarray(X, dtype=np.float64) - ref).reshape(p, -1)
    r = ref.reshape(p, -1)
    per_band = np.linalg.norm(d, axis=1) / np.linalg.norm(r, axis=1)
    assert np.max(per_band) < tol, (int(np.argmax(per_band)), float(np.max(per_band)))
    peak = np.max(np.abs(d), axis=1) / np.max(np.abs(r), axis=1)
    assert np.max(peak) < tol, (int(np.argmax(peak)), float(np.max(peak)))
    # the last row and column (where the symmetric padding is cropped) alone
    H, W = ref.shape[1], ref.shape[2]
    Xa = np.asarray(X, dtype=np.float64)
    for sl in ((slice(None), H - 1, slice(None)), (slice(None), slice(None), W - 1)):
        e = np.linalg.norm(Xa[sl] - ref[sl]) / np.linalg.norm(ref[sl])
        assert e < tol, e


def test_hyres_c0(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    o, X, info, mid = _check_hyres(hyde, c["Y"], 2, 8)
    assert info["rank"] == 4
    T = mid["T"].cpu().numpy()
    assert np.max(np.abs(T - o["T"])) < 1e-4 * np.max(np.abs(o["T"]))


@pytest.mark.parametrize("H,W,p,m,L,r,K,seed", [
    (77, 131, 24, 3, 3, 6, 64, 31),     # ragged: padded to 80 x 136
    (128, 128, 64, 8, 4, 16, 64, 5),    # one cube of the differentiable batch
    (40, 52, 12, 2, 2, 12, 16, 32),     # r_max = p, small K
    (30, 30, 6, 2, 1, 1, 2, 33),        # r_max = 1, K = 2, one level
])
def test_hyres_shapes(hyde, H, W, p, m, L, r, K, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    _check_hyres(hyde, c["Y"], L, r, K)


def test_hyres_c1_full_size(hyde):
    """Houston-shaped 349 x 1905 x 144 cube, 5 levels, r <= 20: the
    benchmark workload, in the launch configuration the benchmark times."""
    c = make_cube(349, 1905, 144, m=12, seed=2)
    o, X, info, mid = _check_hyres(hyde, c["Y"], 5, 20)
    assert O.psnr(c["X"], X) > O.psnr(c["X"], c["Y"]) + 20


def test_hyres_repeat_is_deterministic_in_choice(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    h = hyde.HyRes(32, 64, 64, 2, 8)
    Y = _t(c["Y"])
    X1 = h(Y).clone()
    i1 = h.result_info()
    X2 = h(Y)
    i2 = h.result_info()
    assert (i1["rank"], i1["lambda_index"]) == (i2["rank"], i2["lambda_index"])
    assert O.rel_l2(X2.cpu().numpy(), X1.cpu().numpy()) < 1e-6


def test_hyres_nan_input_sets_status(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    Y = c["Y"].copy()
    Y[3, 10, 10] = np.nan
    h = hyde.HyRes(32, 64, 64, 2, 8)
    h(_t(Y))
    assert h.result_info()["status"] == 3


def test_hyres_rejects_bad_shapes(hyde):
    with pytest.raises(hyde.HydeError):
        hyde.HyRes(32, 64, 64, 2, 40)
    with pytest.raises(hyde.HydeError):
        hyde.HyRes(32, 3, 64, 3, 8)     # padding longer than the image


# ------------------------------------------- per-component thresholds

def _check_hyres_per_component(hyde, Y, L, r_max, K=64, threshold_ll=False):
    """One threshold per kept component. The S table on the GPU may differ
    from the oracle's by a coefficient counted on the other side of a grid
    point (bound of test_sure_table_matches_oracle), so where the oracle's
    choice of k_i (or of the rank) is that close to a runner-up the GPU may
    take the runner-up: its choice must then be a minimiser of the oracle's
    table within that bound, and its estimate must match the oracle run at
    the GPU's choice. Where the choice is clear it must be identical."""
    o = O.hyres(Y, L, r_max, K, lambda_mode="per_component", threshold_ll=threshold_ll)
    p, H, W = Y.shape
    h = hyde.HyRes(p, H, W, L, r_max, K, lambda_mode=hyde.LAMBDA_PER_COMPONENT,
                   threshold_ll=threshold_ll)
    X = h(_t(Y)).cpu().numpy()
    info = h.result_info()
    lam_comp = h.intermediates()["lam_comp"].cpu().numpy().astype(np.float64)
    assert info["status"] == 0
    r = info["rank"]
    assert np.all(lam_comp[r:] == 0.0) and np.all(lam_comp[:r] == lam_comp[:r, :1])
    lams = o["lams"]
    k_gpu = np.rint(lam_comp[:r, 0] / lams[1]).astype(int)
    assert np.allclose(lam_comp[:r, 0], lams[k_gpu], rtol=1e-6, atol=0)
    assert info["lambda_index"] == k_gpu[0]
    S, S_inf = o["S"], o["S_inf"]
    tol = 2.0 * (4.0 + 1e-6 * np.max(np.abs(S)))
    for i in range(r):
        clear = np.all(np.delete(S[i], o["k_comp"][i]) > S[i, o["k_comp"][i]] + tol)
        if clear:
            assert k_gpu[i] == o["k_comp"][i], (i, k_gpu[i], o["k_comp"][i])
        else:
            assert S[i, k_gpu[i]] <= S[i].min() + tol
    U_gpu = S[np.arange(r), k_gpu].sum() + S_inf[r:].sum()
    assert U_gpu <= o["U"].min() + r_max * tol
    if np.all(np.delete(o["U"], o["rank"] - 1) > o["U"].min() + r_max * tol):
        assert r == o["rank"]
    if r == o["rank"] and np.array_equal(k_gpu, o["k_comp"][:r]):
        ref = o["X"]
    else:
        ref = O.hyres(Y, L, r_max, K, rank=r, lam=lams[k_gpu], lambda_mode="per_component",
                      threshold_ll=threshold_ll)["X"]
    err = O.rel_l2(X, ref)
    assert err < REL_L2_PATH, err
    return o, info, k_gpu


def test_hyres_per_component_c0(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    o, info, k_gpu = _check_hyres_per_component(hyde, c["Y"], 2, 8)
    assert info["rank"] == 4
    assert abs(info["sure_min"] - o["U"].min()) < 1e-4 * abs(o["U"].min()) + 8 * 8.0


@pytest.mark.parametrize("H,W,p,m,L,r,K,seed", [
    (77, 131, 24, 3, 3, 6, 64, 31),     # ragged: padded to 80 x 136
    (128, 128, 64, 8, 4, 16, 64, 5),
    (40, 52, 12, 2, 2, 12, 16, 32),     # r_max = p, small K
    (30, 30, 6, 2, 1, 1, 2, 33),        # r_max = 1, K = 2, one level
])
def test_hyres_per_component_shapes(hyde, H, W, p, m, L, r, K, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    _check_hyres_per_component(hyde, c["Y"], L, r, K)


# ------------------------------------- final LL band thresholded too

@pytest.mark.parametrize("H,W,p,m,L,r,K,seed", [
    (64, 64, 32, 4, 2, 8, 64, 1),       # C0: level 2 (with the LL band) in the fused tail
    (77, 131, 24, 3, 3, 6, 64, 31),     # ragged: the scalar level kernel takes the LL band
    (40, 48, 12, 2, 1, 12, 16, 32),     # one level, float4 rows: the register-form kernel
    (349, 256, 144, 12, 5, 20, 64, 2),  # full-cube rows: levels 3-5 fused
    (30, 30, 6, 2, 1, 1, 2, 33),        # one level, unaligned rows, r_max = 1, K = 2
])
def test_hyres_threshold_ll(hyde, H, W, p, m, L, r, K, seed):
    """Every coefficient thresholded (and counted in SURE), the LL band too,
    with the shared threshold and with one per component."""
    c = make_cube(H, W, p, m=m, seed=seed)
    o, X, info, mid = _check_hyres(hyde, c["Y"], L, r, K, threshold_ll=True)
    # the variant changes the table: it is not the default one
    o0 = O.hyres(c["Y"], L, r, K)
    assert not np.allclose(o["S"], o0["S"])
    _check_hyres_per_component(hyde, c["Y"], L, r, K, threshold_ll=True)


def test_hyres_scaled_rejects_per_component(hyde):
    g = hyde.HyResGrad(32, 64, 64, 2, 8)
    g.params.lambda_mode = hyde.LAMBDA_PER_COMPONENT
    s = torch.ones(8, 2, dtype=torch.float32, device="cuda")
    with pytest.raises(hyde.HydeError):
        g.forward_scaled(_t(make_cube(64, 64, 32, m=4, seed=1)["Y"]), s)


# ------------------------------------------------------ host cube stream

@pytest.mark.parametrize("count", [1, 3, 4])
def test_denoise_host_stream_matches_device_calls(hyde, count):
    """hyde_hyres_denoise_host (copies of cube s+1 in and s-1 out overlapping
    the denoise of cube s, device buffers reused in turn) gives each cube the
    result and the (rank, lambda) choice of a plain device call."""
    cubes = [make_cube(64, 64, 32, m=4, seed=40 + s)["Y"] for s in range(count)]
    h = hyde.HyRes(32, 64, 64, 2, 8)
    refs, choices = [], []
    for Y in cubes:
        refs.append(h(_t(Y)).cpu().numpy())
        info = h.result_info()
        choices.append((info["rank"], info["lambda_index"]))
    Ys = [torch.from_numpy(Y).pin_memory() for Y in cubes]
    Xs = [torch.full_like(Ys[0], float("nan")).pin_memory() for _ in cubes]
    nb = hyde.INFO_BYTES
    infos = torch.zeros(count * nb, dtype=torch.uint8).pin_memory()
    h.denoise_host(Ys, Xs, infos)
    torch.cuda.synchronize()
    for s in range(count):
        assert O.rel_l2(Xs[s].numpy(), refs[s]) < 1e-6
        info = hyde.parse_info(infos[s * nb:(s + 1) * nb])
        assert info["status"] == 0
        assert (info["rank"], info["lambda_index"]) == choices[s]


# ---------------------------------------------- per-level thresholds

def _check_hyres_per_level(hyde, Y, L, r_max, K=64, threshold_ll=False):
    """One threshold per (kept component, level): the device's choice on its
    own tables, its tables and choices on the separated components, and its
    estimate at its own choice, against the oracle (selection_checks)."""
    o = O.hyres(Y, L, r_max, K, lambda_mode="per_level", threshold_ll=threshold_ll)
    p, H, W = Y.shape
    h = hyde.HyRes(p, H, W, L, r_max, K, lambda_mode=hyde.LAMBDA_PER_LEVEL,
                   threshold_ll=threshold_ll)
    X = h(_t(Y)).cpu().numpy()
    info = h.result_info()
    mid = h.intermediates()
    assert info["status"] == 0
    assert tuple(mid["S"].shape) == (r_max, L, K)
    check_per_level_choice(
        o, Y.shape, L, r_max, threshold_ll, coef_dev=mid["coef"].cpu().numpy(),
        S_dev=mid["S"].cpu().numpy(), S_inf_dev=mid["S_inf"].cpu().numpy(),
        rank=info["rank"], lam=mid["lam_comp"].cpu().numpy().astype(np.float64),
        sure_min=info["sure_min"], lambda_index=info["lambda_index"], X=X, Y=Y)
    return o, info


def test_hyres_per_level_c0(hyde):
    c = make_cube(64, 64, 32, m=4, seed=1)
    o, info = _check_hyres_per_level(hyde, c["Y"], 2, 8)
    assert info["rank"] == 4


@pytest.mark.parametrize("H,W,p,m,L,r,K,seed", [
    (77, 131, 24, 3, 3, 6, 64, 31),     # ragged: padded to 80 x 136
    (128, 128, 64, 8, 4, 16, 64, 5),
    (40, 52, 12, 2, 2, 12, 16, 32),     # r_max = p, small K
    (30, 30, 6, 2, 1, 1, 2, 33),        # r_max = 1, K = 2, one level
])
def test_hyres_per_level_shapes(hyde, H, W, p, m, L, r, K, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    _check_hyres_per_level(hyde, c["Y"], L, r, K)


@pytest.mark.parametrize("H,W,p,m,L,r,K,seed", [
    (64, 64, 32, 4, 2, 8, 64, 1),
    (349, 256, 144, 12, 5, 20, 64, 2),
])
def test_hyres_per_level_threshold_ll(hyde, H, W, p, m, L, r, K, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    _check_hyres_per_level(hyde, c["Y"], L, r, K, threshold_ll=True)
