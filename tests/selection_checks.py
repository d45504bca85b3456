"""Checks of a per-(component, level) threshold choice made on the device
against the FP64 oracle. Shared by the GPU parity tests and by a CPU test of
the checks themselves (run on an oracle whose eigenbasis was computed in
float32, the perturbation a float32 device path brings).

What is compared, and why:
- the choice on the device's own SURE tables must be exactly what the
  oracle's selection function makes of those tables (this pins the
  selection arithmetic, whatever the tables are);
- the tables and the choices are compared with the oracle's only for the
  leading components that are well separated in eigenvalue: past them the
  components lie in the near-degenerate noise cluster, whose split into
  single eigenvectors a float32 and a float64 solver make differently, so
  their per-component tables legitimately differ (by 2-14 at 349 x 256 x 144
  under a float32 basis alone);
- the estimate is compared with the oracle run at the device's choice, to
  1e-5 while the kept rank stays among the separated components and to 1e-3
  once it reaches into the cluster (the rule the window tests follow).
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


def check_per_level_choice(o, shape, L, r_max, threshold_ll, *, S_dev, S_inf_dev, rank,
                           lam, sure_min, lambda_index, X, Y):
    """``o``: the oracle's per-level run on ``Y``; the keyword arguments are
    what the device reported: its SURE tables ``S_dev[r_max][L][K]`` and
    ``S_inf_dev[r_max]``, the rank, the threshold table ``lam[r_max][L]``,
    the info record's ``sure_min`` and ``lambda_index``, and the estimate.
    Returns the number of separated leading components."""
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
    # tables and choices on the separated components
    n_sep = separated_prefix(o["evals"])
    ns = min(n_sep, r_max)
    S_lev = o["S_lev"]
    tol = 2.0 * (4.0 + 1e-6 * np.max(np.abs(S_lev)))
    if ns:
        assert np.max(np.abs(S_dev[:ns] - S_lev[:ns])) < tol
    for i in range(min(r, ns)):
        for l in range(L):
            kr = o["k_lev"][i, l]
            if np.all(np.delete(S_lev[i, l], kr) > S_lev[i, l, kr] + tol):
                assert k_dev[i, l] == kr, (i, l, k_dev[i, l], kr)
            else:
                assert S_lev[i, l, k_dev[i, l]] <= S_lev[i, l].min() + tol
    # the rank, where every kept component is separated on both sides
    if r <= n_sep and o["rank"] <= n_sep:
        U_dev = sum(n_kept + S_lev[i, np.arange(L), k_dev[i]].sum() for i in range(r))
        U_dev += o["S_inf"][r:].sum()
        assert U_dev <= o["U"].min() + r_max * L * tol
        if np.all(np.delete(o["U"], o["rank"] - 1) > o["U"].min() + r_max * L * tol):
            assert r == o["rank"]
    # the estimate at the device's choice
    if r == o["rank"] and np.array_equal(k_dev, o["k_lev"][:r]):
        ref = o["X"]
    else:
        ref = O.hyres(Y, L, r_max, K, rank=r, lam=lams[k_dev], lambda_mode="per_level",
                      threshold_ll=threshold_ll)["X"]
    err = O.rel_l2(X, ref)
    assert err < (REL_L2_SEPARATED if r <= n_sep else REL_L2_CLUSTER), err
    return n_sep
