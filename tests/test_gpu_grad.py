"""GPU parity of the differentiation form (learnable per-(component, level)
threshold scales) against the FP64 oracle: forward with scales, the
hand-written adjoint for a given dL/dX, the SURE loss and its gradient, and
the torch.autograd wrappers against central finite differences."""

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_cube

pytestmark = pytest.mark.gpu


def _t(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


CASES = [
    # H, W, p, m, L, r_max, seed: the differentiable-batch cube shape, and a
    # ragged one that needs padding
    (128, 128, 64, 8, 4, 16, 5),
    (77, 90, 24, 3, 3, 8, 61),
]


def _scale(rows, L, seed):
    rng = np.random.default_rng(seed)
    return (1.0 + 0.2 * rng.standard_normal((rows, L))).astype(np.float32)


def _flip_allowance(o, L, s, rel=1e-5):
    """The a.e. SURE gradient 2 lam* lam_il #{|c| > lam_il} is piecewise
    constant in the coefficients: each detail coefficient that float
    arithmetic may put on the other side of its threshold (the oracle's lies
    within ``rel`` of it) can move entry (i, l) by 2 lam* lam_il."""
    r = o["rank"]
    C, lev = o["C"][:r], o["level_map"]
    allow = np.zeros(s.shape, dtype=np.float64)
    for i in range(r):
        for l in range(1, L + 1):
            lam = o["lam"] * float(s[i, l - 1])
            c = np.abs(C[i][lev == l])
            near = np.count_nonzero(np.abs(c - lam) <= rel * lam)
            allow[i, l - 1] = near * 2.0 * o["lam"] * lam
    return allow


@pytest.mark.parametrize("H,W,p,m,L,r,seed", CASES)
def test_scaled_forward_matches_oracle(hyde, H, W, p, m, L, r, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    s = _scale(p, L, seed)
    o = O.hyres_scaled(c["Y"], L, r, s.astype(np.float64))
    g = hyde.HyResGrad(p, H, W, L, r)
    X = g.forward_scaled(_t(c["Y"]), _t(s)).cpu().numpy()
    info = g.result_info()
    assert (info["rank"], info["lambda_index"]) == (o["rank"], o["k"])
    assert O.rel_l2(X, o["X_scaled"]) < 1e-5


@pytest.mark.parametrize("H,W,p,m,L,r,seed", CASES)
def test_mse_adjoint_matches_oracle(hyde, H, W, p, m, L, r, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    s = _scale(p, L, seed + 1)
    o = O.hyres_scaled(c["Y"], L, r, s.astype(np.float64))
    G = (2.0 * (o["X_scaled"] - c["X"]) / c["X"].size).astype(np.float32)
    ref, _ = O.hyres_scaled_grad(c["Y"], G.astype(np.float64), L, r, s.astype(np.float64))
    g = hyde.HyResGrad(p, H, W, L, r)
    Y = _t(c["Y"])
    g.forward_scaled(Y, _t(s))
    ds = g.backward_scaled(Y, _t(G), _t(s), loss=0).cpu().numpy()
    rk = o["rank"]
    assert np.all(ds[rk:] == 0)
    # float32 adjoint (projection, DWT) against FP64; a coefficient within
    # rounding of its threshold may flip the mask (one term of a large sum)
    assert np.linalg.norm(ds[:rk] - ref[:rk]) <= 1e-4 * np.linalg.norm(ref[:rk])


@pytest.mark.parametrize("H,W,p,m,L,r,seed", CASES)
def test_sure_loss_and_gradient_match_oracle(hyde, H, W, p, m, L, r, seed):
    c = make_cube(H, W, p, m=m, seed=seed)
    s = _scale(p, L, seed + 2)
    o = O.hyres_scaled(c["Y"], L, r, s.astype(np.float64))
    val, ref = O.sure_loss_scaled(o, L, s.astype(np.float64))
    g = hyde.HyResGrad(p, H, W, L, r)
    Y = _t(c["Y"])
    g.forward_scaled(Y, _t(s))
    ds = g.backward_scaled(Y, None, _t(s), loss=1).cpu().numpy()
    got = float(g.sure_value.item())
    rk = o["rank"]
    assert abs(got - val) <= 1e-5 * abs(val) + 8.0
    allow = _flip_allowance(o, L, s)
    assert np.linalg.norm(ds[:rk] - ref[:rk]) <= (1e-4 * np.linalg.norm(ref[:rk]) +
                                                  np.linalg.norm(allow[:rk]))


def test_autograd_mse_against_finite_differences(hyde):
    H, W, p, m, L, r, seed = 96, 96, 32, 4, 3, 8, 71
    c = make_cube(H, W, p, m=m, seed=seed)
    Y = _t(c["Y"])
    Xc = _t(c["X"])
    g = hyde.HyResGrad(p, H, W, L, r)
    s0 = torch.from_numpy(_scale(p, L, 3)).cuda()

    def loss_of(s):
        return torch.mean((hyde.hyres_scaled(Y, s, g) - Xc) ** 2)

    s = s0.clone().requires_grad_(True)
    loss = loss_of(s)
    loss.backward()
    grad = s.grad.detach().cpu().numpy()
    rk = g.result_info()["rank"]
    h = 1e-3
    fd = np.zeros_like(grad)
    with torch.no_grad():
        for i in range(rk):
            for l in range(L):
                e = torch.zeros_like(s0)
                e[i, l] = h
                fd[i, l] = (loss_of(s0 + e).item() - loss_of(s0 - e).item()) / (2 * h)
    # raw differences include coefficients crossing their threshold: ~1 %
    assert np.linalg.norm(fd[:rk] - grad[:rk]) <= 2e-2 * np.linalg.norm(grad[:rk])
    assert np.all(grad[rk:] == 0)


def test_autograd_sure_loss_and_batch_sum(hyde):
    """A batch of cubes: the gradient of the summed loss is the sum of the
    per-cube oracle gradients."""
    H, W, p, L, r = 64, 64, 16, 3, 6
    cubes = [make_cube(H, W, p, m=3, seed=80 + b) for b in range(3)]
    models = [hyde.HyResGrad(p, H, W, L, r) for _ in cubes]
    s = torch.full((p, L), 1.05, device="cuda", requires_grad=True)
    total = sum(hyde.hyres_sure_loss(_t(cb["Y"]), s, mdl) for cb, mdl in zip(cubes, models))
    total.backward()
    ref_val, ref_grad = 0.0, np.zeros((p, L))
    for cb in cubes:
        o = O.hyres_scaled(cb["Y"], L, r, np.full((p, L), 1.05))
        v, gr = O.sure_loss_scaled(o, L, np.full((p, L), 1.05))
        ref_val += v
        ref_grad += gr
    assert abs(total.item() - ref_val) <= 1e-5 * abs(ref_val) + 24.0
    got = s.grad.cpu().numpy()
    assert np.linalg.norm(got - ref_grad) <= 1e-4 * np.linalg.norm(ref_grad)


def test_batched_streams_match_sequential(hyde):
    """The batch on one stream per cube gives the same outputs and the same
    summed gradient as the cubes one after another."""
    H, W, p, L, r = 64, 64, 16, 3, 6
    cubes = [make_cube(H, W, p, m=3, seed=90 + b) for b in range(4)]
    Ys = [_t(cb["Y"]) for cb in cubes]
    Xc = [_t(cb["X"]) for cb in cubes]
    s0 = torch.from_numpy(_scale(p, L, 9)).cuda()

    seq_models = [hyde.HyResGrad(p, H, W, L, r) for _ in cubes]
    s_seq = s0.clone().requires_grad_(True)
    outs_seq = [hyde.hyres_scaled(Y, s_seq, m) for Y, m in zip(Ys, seq_models)]
    sum(torch.mean((X - C) ** 2) for X, C in zip(outs_seq, Xc)).backward()

    bat_models = [hyde.HyResGrad(p, H, W, L, r) for _ in cubes]
    s_bat = s0.clone().requires_grad_(True)
    outs_bat = hyde.hyres_scaled_batch(Ys, s_bat, bat_models)
    sum(torch.mean((X - C) ** 2) for X, C in zip(outs_bat, Xc)).backward()
    torch.cuda.synchronize()

    for a, b in zip(outs_seq, outs_bat):
        assert O.rel_l2(b.detach().cpu().numpy(), a.detach().cpu().numpy()) < 1e-6
    gs, gb = s_seq.grad.cpu().numpy(), s_bat.grad.cpu().numpy()
    assert np.linalg.norm(gb - gs) <= 1e-5 * np.linalg.norm(gs)
