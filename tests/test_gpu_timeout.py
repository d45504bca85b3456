"""The bounded waits of the tensor-core Gram kernels run out, on purpose.

Every mbarrier wait inside the tcgen05 Gram kernels (split-BF16 and
split-TF32) is bounded in time. Here
the limit of its main-loop waits is set to 1 ns (``hyde_set_wait_limit_ns``),
so the tensor-core issuer gives up at its first wait, before the loaders have
filled a stage, and the loaders (and, in the split-TF32 kernel, the TMA
warp and the TMEM drain warps) give up when a stage is never released. The
kernel must then report HYDE_ERR_TIMEOUT through the device status word,
leave its output zero, free its tensor memory and return, and the CUDA
context must stay usable: with the default limit restored the same call
succeeds and matches the plain FP32 path. No wait here depends on a flag
that nothing sets for longer than the limit, and no fault is raised.
"""

import numpy as np
import pytest
import torch

import oracle as O
from synth import make_cube

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["bf16x3", "tf32x3"])
def test_tensor_core_gram_timeout_is_reported_and_recovers(hyde, prec):
    from paper_2204_06979_gb300 import _lib
    lib = _lib.load()
    c = make_cube(349, 256, 144, m=12, seed=2)
    Y = torch.from_numpy(c["Y"]).cuda()
    p, H, W = c["Y"].shape
    precision = hyde.PREC_BF16X3 if prec == "bf16x3" else hyde.PREC_TF32X3
    h = hyde.HyRes(p, H, W, 5, 20, precision=precision)
    prev = lib.hyde_set_wait_limit_ns(1)
    try:
        h(Y)
        torch.cuda.synchronize()
        info = h.result_info()
    finally:
        lib.hyde_set_wait_limit_ns(prev)
    assert info["status"] == 5            # HYDE_ERR_TIMEOUT, not a fault
    R = h.intermediates()["R"].cpu().numpy()
    assert np.all(R == 0.0)               # every CTA gave up before adding anything
    # the context is intact: the same call with the default limit succeeds
    X = h(Y)
    torch.cuda.synchronize()
    assert h.result_info()["status"] == 0
    ref = hyde.HyRes(p, H, W, 5, 20)(Y)
    torch.cuda.synchronize()
    assert O.rel_l2(X.cpu().numpy(), ref.cpu().numpy()) < 1e-4
