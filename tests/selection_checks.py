"""Checks of a per-(component, level) threshold choice made on the device
against the FP64 oracle. Shared by the GPU parity tests and by a CPU test of
the checks themselves (run on an oracle whose eigenbasis was computed in
float32, the perturbation a float32 device path brings).

What is compared, and why:
- the device's SURE tables must be those of its own coefficients (the
  oracle's tables of the float32 coefficients the device left in its
  workspace), to the bound of the histogram's rounding at grid points: this
  pins the binning, the level groups and the table arithmetic. Against the
  oracle's FP64 coefficients the tables legitimately differ by more: a group
  of 67k coefficients with a relative error of ~2e-5 (the noise estimate's)
  has tens of coefficients within that error of a grid point, and past the
  separated components the noise cluster's split into single eigenvectors
  differs between float32 and float64 solvers;
- the choice on the device's tables must be exactly what the oracle's
  selection function makes of those tables;
- the estimate is compared with the oracle run at the device's choice, to
  1e-5 while the kept rank stays among the components whose eigenvalues are
  separated and to 1e-3 once it reaches into the cluster (the rule the
  window tests follow).
"""

import numpy as np

import oracle as O

REL_L2_SEPARATED = 1e-5
REL_L2_CLUSTER = 1e-3


def separated_prefix(evals, rel_gap=0.05):
    """Number of leading components each of which exceeds the next
    eigenvalue by more than ``rel_gap`` (relative)."""
    n = 0
    while n + 1 < len(evals) and evals[n] > (1.0 + rel_gap) * evals[n + 1]:
        n += 1
    return n


def check_per_level_choice(o, shape, L, r_max, threshold_ll, *, coef_dev, S_dev, S_inf_dev,
                           rank, lam, sure_min, lambda_index, X, Y):
    """``o``: the oracle's per-level run on ``Y``; the keyword arguments are
    what the device reported: its wavelet coefficients
    ``coef_dev[r_max][Hp][Wp]`` (float32), SURE tables ``S_dev[r_max][L][K]``
    and ``S_inf_dev[r_max]``, the rank, the threshold table
    ``lam[r_max][L]``, the info record's ``sure_min`` and ``lambda_index``,
    and the estimate. Returns the number of separated leading components."""
    p, H, W = shape
    K = len(o["lams"])
    lams = o["lams"]
    Hp, Wp = O.padded_shape(H, W, L)
    n_kept = 0 if threshold_ll else (Hp >> L) * (Wp >> L)
    r = int(rank)
    assert 1 <= r <= r_max
    # the threshold table: grid values on the kept rows, zero elsewhere
    assert np.all(lam[r:] == 0.0)
    k_dev = np.rint(lam[:r] / lams[1]).astype(int)
    assert np.all((k_dev >= 0) & (k_dev < K))
    assert np.allclose(lam[:r], lams[k_dev], rtol=1e-6, atol=0)
    assert lambda_index == k_dev[0, 0]
    # the selection on the device's own tables
    r2, k2, U2, _ = O.select_rank_lambda_per_level(S_dev, S_inf_dev, n_kept)
    assert r2 == r, (r2, r)
    assert np.array_equal(k2[:r], k_dev)
    assert abs(U2.min() - sure_min) <= 1e-9 * max(abs(U2.min()), 1.0)
    # the device's tables are those of its own coefficients (a coefficient
    # within rounding of a grid point may land in either bin: about 2 each)
    C = np.asarray(coef_dev, dtype=np.float64)
    S_ref = O.sure_table_levels(C, L, lams, threshold_ll)
    assert np.max(np.abs(S_dev - S_ref)) < 4.0 + 1e-6 * np.max(np.abs(S_ref))
    Sinf_ref = np.sum(C * C, axis=(1, 2)) - Hp * Wp
    # sums of squares: float per thread on the device, double across blocks
    assert np.max(np.abs(S_inf_dev - Sinf_ref)) < 1e-5 * np.max(np.abs(Sinf_ref)) + 1e-3
    n_sep = separated_prefix(o["evals"])
    # the estimate at the device's choice
    if r == o["rank"] and np.array_equal(k_dev, o["k_lev"][:r]):
        ref = o["X"]
    else:
        ref = O.hyres(Y, L, r_max, K, rank=r, lam=lams[k_dev], lambda_mode="per_level",
                      threshold_ll=threshold_ll)["X"]
    err = O.rel_l2(X, ref)
    assert err < (REL_L2_SEPARATED if r <= n_sep else REL_L2_CLUSTER), err
    return n_sep
