"""The allocation-free Gram entry point against the regular one and the
FP64 oracle.

``hyde_gram_noalloc`` serves callers that cannot hand the library a
workspace because they may not allocate device memory themselves: code
embedded in a host framework that owns every device allocation, or a loop
with a fixed memory budget that must not allocate. It keeps its partial sums
in one fixed array in device memory instead of a caller workspace.

This file is collected last on purpose, so a run that stops at the first
failure has already run every other test; it also passes on its own in a
fresh process.
"""

import ctypes

import numpy as np
import pytest
import torch

import oracle as O

pytestmark = pytest.mark.gpu


def _gram_via_workspace(lib, Y, p, n):
    sz = ctypes.c_size_t()
    assert lib.hyde_gram_workspace_size(p, n, 0, ctypes.byref(sz)) == 0
    ws = torch.empty(max(sz.value, 256), dtype=torch.uint8, device="cuda")
    R = torch.empty((p, p), dtype=torch.float64, device="cuda")
    code = lib.hyde_gram(Y.data_ptr(), p, n, 0, R.data_ptr(), ws.data_ptr(), ws.numel(),
                         torch.cuda.current_stream().cuda_stream)
    assert code == 0
    return R


@pytest.mark.parametrize("p,H,W", [(144, 349, 1905), (256, 96, 97), (37, 33, 51)])
def test_gram_noalloc_matches_workspace_gram_twice(p, H, W):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_06979_gb300 import _lib
    lib = _lib.load()
    assert lib.hyde_gram_noalloc_scratch_bytes() == 16 << 20
    rng = np.random.default_rng(p * 7 + H)
    Y = torch.from_numpy((rng.standard_normal((p, H, W)) + 0.25).astype(np.float32)).cuda()
    n = H * W
    ref = _gram_via_workspace(lib, Y, p, n).cpu().numpy()
    exact = O.gram(Y.cpu().numpy())
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(2):   # the shared array keeps the previous call's contents
        R = torch.full((p, p), np.nan, dtype=torch.float64, device="cuda")
        assert lib.hyde_gram_noalloc(Y.data_ptr(), p, n, R.data_ptr(), stream) == 0
        got = R.cpu().numpy()
        assert np.all(np.isfinite(got))
        # same tolerance as the Gram parity tests: float partial sums
        assert np.max(np.abs(got - ref)) < 2e-6 * np.max(np.abs(ref))
        # and the same bound against the FP64 oracle's Y^T Y
        assert np.max(np.abs(got - exact)) < 2e-6 * np.max(np.abs(exact))


def test_gram_noalloc_rejects_bad_arguments():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2204_06979_gb300 import _lib
    lib = _lib.load()
    R = torch.empty((4, 4), dtype=torch.float64, device="cuda")
    assert lib.hyde_gram_noalloc(None, 4, 100, R.data_ptr(), None) == 1
    Y = torch.zeros((300, 10), dtype=torch.float32, device="cuda")
    assert lib.hyde_gram_noalloc(Y.data_ptr(), 300, 10, R.data_ptr(), None) == 2
