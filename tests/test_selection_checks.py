"""CPU test of the per-level checks that the GPU parity tests apply
(``selection_checks``): they accept what a float32 eigenbasis legitimately
changes, both below the noise cluster and with the kept rank inside it, and
they reject planted mistakes in the device's tables, thresholds or
estimate."""

import numpy as np
import pytest

import oracle as O
from selection_checks import check_per_level_choice, separated_prefix
from synth import make_cube

CASES = {
    # 128 x 128 x 64, 8 endmembers: rank 7, components 7.. in the noise cluster
    "below_cluster": dict(shape=(64, 128, 128), m=8, L=4, r_max=16, seed=5, threshold_ll=False),
    # 349 x 256 x 144 with the LL band thresholded: rank 20 = r_max, inside the cluster
    "into_cluster": dict(shape=(144, 349, 256), m=12, L=5, r_max=20, seed=2, threshold_ll=True),
}


def _runs(case):
    c = CASES[case]
    p, H, W = c["shape"]
    Y = make_cube(H, W, p, m=c["m"], seed=c["seed"])["Y"]
    o = O.hyres(Y, c["L"], c["r_max"], 64, lambda_mode="per_level",
                threshold_ll=c["threshold_ll"])
    # the stand-in device: the same path on an eigenbasis computed in float32
    _, V = np.linalg.eigh(o["Rw"].astype(np.float32))
    V = V[:, ::-1][:, : c["r_max"]].astype(np.float64)
    V *= np.sign(np.sum(V * o["V"], axis=0))
    d = O.hyres(Y, c["L"], c["r_max"], 64, V=V, lambda_mode="per_level",
                threshold_ll=c["threshold_ll"])
    return c, Y, o, d


def _device_args(d, c):
    r = d["rank"]
    lam = np.zeros((c["r_max"], c["L"]))
    lam[:r] = d["lam_comp"].astype(np.float32)
    return dict(coef_dev=d["C"].astype(np.float32), S_dev=d["S_lev"].copy(),
                S_inf_dev=d["S_inf"].copy(), rank=r, lam=lam,
                sure_min=float(d["U"].min()), lambda_index=int(d["k_lev"][0, 0]),
                X=d["X"].copy())


def _check(c, Y, o, args):
    return check_per_level_choice(o, Y.shape, c["L"], c["r_max"], c["threshold_ll"], Y=Y,
                                  **args)


def test_separated_prefix():
    assert separated_prefix([10.0, 5.0, 1.01, 1.0]) == 2
    assert separated_prefix([1.0, 1.0, 1.0]) == 0
    assert separated_prefix([3.0, 1.0]) == 1


@pytest.mark.parametrize("case", sorted(CASES))
def test_checks_accept_a_float32_basis(case):
    c, Y, o, d = _runs(case)
    n_sep = _check(c, Y, o, _device_args(d, c))
    if case == "below_cluster":
        assert o["rank"] <= n_sep
    else:
        assert o["rank"] > n_sep


@pytest.mark.parametrize("case", sorted(CASES))
def test_checks_reject_planted_mistakes(case):
    c, Y, o, d = _runs(case)
    base = _device_args(d, c)
    # a threshold that is not the minimiser of its own table
    bad = dict(base, lam=base["lam"].copy())
    K = len(o["lams"])
    k00 = int(d["k_lev"][0, 0])
    bad["lam"][0, 0] = np.float32(o["lams"][(k00 + 7) % K])
    bad["lambda_index"] = (k00 + 7) % K
    with pytest.raises(AssertionError):
        _check(c, Y, o, bad)
    # a table row off by a dropped term, in a leading and in a cluster component
    for i in (0, c["r_max"] - 1):
        bad = dict(base, S_dev=base["S_dev"].copy())
        bad["S_dev"][i, c["L"] - 1] += 12.0
        with pytest.raises(AssertionError):
            _check(c, Y, o, bad)
    # coefficients of one level binned into the next level's group
    bad = dict(base, S_dev=base["S_dev"].copy())
    bad["S_dev"][:, [0, 1]] = bad["S_dev"][:, [1, 0]]
    with pytest.raises(AssertionError):
        _check(c, Y, o, bad)
    # an estimate off by 2e-3 (relative), above both tolerances
    rng = np.random.default_rng(3)
    noise = rng.standard_normal(base["X"].shape)
    bad = dict(base, X=base["X"] + 2e-3 * np.linalg.norm(base["X"]) / np.linalg.norm(noise)
               * noise)
    with pytest.raises(AssertionError):
        _check(c, Y, o, bad)
