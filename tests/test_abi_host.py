"""Host-side checks of the C ABI that need no GPU: the library builds and
loads, exports every function include/hyde.h declares, and rejects bad
arguments before touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "hyde.h")


def _declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hyde_[a-z0-9_]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_2204_06979_gb300 import build, _lib
    build.build()
    return _lib.load()


def test_header_declares_the_boundary():
    names = _declared_functions()
    for must in ("hyde_noise_est", "hyde_dwt2", "hyde_idwt2", "hyde_gram",
                 "hyde_hyres_denoise", "hyde_workspace_size", "hyde_sure_table",
                 "hyde_eig_sym_top"):
        assert must in names


def test_library_exports_every_declared_symbol(lib):
    from paper_2204_06979_gb300 import _lib
    for name in _declared_functions():
        assert hasattr(lib, name), name
        assert name in _lib.SIGNATURES, f"binding lacks a signature for {name}"


def test_status_strings_and_version(lib):
    assert lib.hyde_version() >= 100
    for code in range(8):
        assert lib.hyde_status_string(code)
    assert lib.hyde_status_string(99) == b"unknown status"


def test_kernel_launch_count(lib):
    """The launch count the benchmark reports: gram 2, noise 2, eig 3,
    weights 1, projection 1, SURE 2, back-projection 1, and per direction one
    DWT launch per level except that the coarse levels (those whose LL band
    has at most 12288 values, when the quarter-width stays a multiple of 4)
    run as one fused launch."""
    from paper_2204_06979_gb300 import api
    def count(p, H, W, L, r):
        prm = api.params(L, r)
        return lib.hyde_hyres_kernel_launches(p, H, W, ctypes.byref(prm))
    assert count(144, 349, 1905, 5, 20) == 12 + 2 * 4   # levels 1-3, then 4-5 fused
    assert count(32, 64, 64, 2, 8) == 12 + 2 * 2       # level 1, then 2 fused
    assert count(24, 77, 131, 3, 6) == 12 + 2 * 3      # 136 / 8 = 17: no fused tail
    assert count(32, 64, 64, 11, 8) == -1
    assert lib.hyde_hyres_kernel_launches(32, 64, 64, None) == -1


def test_grid_sm_cap_setter(lib):
    """hyde_set_grid_sm_cap returns the previous cap; 0 (or less) removes it."""
    prev = lib.hyde_set_grid_sm_cap(10)
    assert prev == 0
    assert lib.hyde_set_grid_sm_cap(19) == 10
    assert lib.hyde_set_grid_sm_cap(-3) == 19
    assert lib.hyde_set_grid_sm_cap(0) == 0


def test_bad_arguments_rejected_on_host(lib):
    from paper_2204_06979_gb300._lib import HydeParams
    sz = ctypes.c_size_t()
    # DWT: padding longer than the image, bad batch, bad levels
    assert lib.hyde_dwt_workspace_size(1, 3, 40, 3, ctypes.byref(sz)) == 2
    assert lib.hyde_dwt_workspace_size(0, 32, 32, 2, ctypes.byref(sz)) == 2
    assert lib.hyde_dwt_workspace_size(1, 32, 32, 11, ctypes.byref(sz)) == 2
    assert lib.hyde_dwt_workspace_size(1, 32, 32, 2, None) == 1
    # DWT with null pointers / wrong wavelet
    assert lib.hyde_dwt2(None, None, 1, 32, 32, 2, 2, None, 0, None) == 1
    assert lib.hyde_dwt2(1, 2, 1, 32, 32, 4, 2, None, 0, None) == 1
    # SURE sizes
    assert lib.hyde_sure_workspace_size(1, 1, ctypes.byref(sz)) == 2
    assert lib.hyde_sure_workspace_size(1, 300, ctypes.byref(sz)) == 2
    # whole path: invalid params
    p = HydeParams()
    p.wavelet, p.levels, p.r_max, p.n_lambda, p.precision = 2, 2, 8, 64, 0
    assert lib.hyde_hyres_denoise(None, None, 32, 64, 64, ctypes.byref(p), None, None, 0, None) == 1
    p.wavelet = 3
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 1
    p.wavelet, p.r_max = 2, 40
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 2
    p.r_max, p.n_lambda = 8, 1
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 2
    p.n_lambda, p.reserved = 64, 1
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 1
    p.reserved = 0
    p.threshold_ll = 2
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 1
    p.threshold_ll = 0
    assert lib.hyde_workspace_size(1, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 2
    p.lambda_mode = 3
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(p), ctypes.byref(sz)) == 1
    p.lambda_mode = 0
    assert lib.hyde_eig_sym_top(None, 4, 2, None, None, None, None, 0, None) == 1
    sz = ctypes.c_size_t()
    assert lib.hyde_eig_workspace_size(4, 2, None) == 1
    assert lib.hyde_eig_workspace_size(1, 1, ctypes.byref(sz)) == 2     # one band
    assert lib.hyde_eig_workspace_size(8, 9, ctypes.byref(sz)) == 2     # r > p
    assert lib.hyde_eig_workspace_size(64, 33, ctypes.byref(sz)) == 2   # r > 32
    assert lib.hyde_eig_workspace_size(144, 20, ctypes.byref(sz)) == 0
    assert sz.value >= (144 * 144 + 20 * 144) * 4
    # a workspace that is missing or too small is refused before any launch
    assert lib.hyde_eig_sym_top(1, 144, 20, 1, 1, None, None, 0, None) == 7
    assert lib.hyde_eig_sym_top(1, 144, 20, 1, 1, None, 256, 1024, None) == 7


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2204_06979_gb300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_LIB", None)
    with pytest.raises(ImportError):
        _lib.load()


def test_lambda_mode_params(lib):
    """Per-component thresholds and the thresholded LL band are rejected,
    before any device query, by the scaled (differentiation) entry points,
    and an unknown mode by every entry point."""
    from paper_2204_06979_gb300 import api
    comp = api.params(3, 8, 64, lambda_mode=api.LAMBDA_PER_COMPONENT)
    bad = api.params(3, 8, 64, lambda_mode=5)
    sz = ctypes.c_size_t()
    assert lib.hyde_backward_workspace_size(32, 64, 64, ctypes.byref(comp), ctypes.byref(sz)) == 1
    assert lib.hyde_hyres_denoise_scaled(1, 2, 32, 64, 64, ctypes.byref(comp), 3, None, 4,
                                         1 << 30, None) == 1
    assert lib.hyde_workspace_size(32, 64, 64, ctypes.byref(bad), ctypes.byref(sz)) == 1
    assert lib.hyde_hyres_kernel_launches(32, 64, 64, ctypes.byref(bad)) == -1
    # per-level histograms that would not fit in shared memory
    big = api.params(10, 8, 256, lambda_mode=api.LAMBDA_PER_LEVEL)
    assert lib.hyde_workspace_size(32, 1024, 1024, ctypes.byref(big), ctypes.byref(sz)) == 2
    lvl = api.params(3, 8, 64, lambda_mode=api.LAMBDA_PER_LEVEL)
    assert lib.hyde_backward_workspace_size(32, 64, 64, ctypes.byref(lvl), ctypes.byref(sz)) == 1
    # the final LL band thresholded too: likewise only outside the scaled forms
    ll = api.params(3, 8, 64, threshold_ll=True)
    assert lib.hyde_backward_workspace_size(32, 64, 64, ctypes.byref(ll), ctypes.byref(sz)) == 1
    assert lib.hyde_hyres_denoise_scaled(1, 2, 32, 64, 64, ctypes.byref(ll), 3, None, 4,
                                         1 << 30, None) == 1


def test_remaining_entry_points_reject_bad_arguments_on_host(lib):
    """Every entry point not covered above rejects null pointers, bad sizes
    and bad shapes before any device query (status codes: 1 invalid
    argument, 2 unsupported shape)."""
    from paper_2204_06979_gb300 import api
    from paper_2204_06979_gb300._lib import HydeWindow, HydeWsLayout
    sz = ctypes.c_size_t()
    prm = api.params(2, 8, 64)
    # Gram workspace: no output, an unknown precision
    assert lib.hyde_gram_workspace_size(32, 4096, 0, None) == 1
    assert lib.hyde_gram_workspace_size(32, 4096, 9, ctypes.byref(sz)) == 1
    assert lib.hyde_gram_workspace_size(32, 0, 2, ctypes.byref(sz)) == 2
    # split-TF32 Gram: p a multiple of 4 and at most 160, checked before any device query
    assert lib.hyde_gram_workspace_size(37, 4096, 1, ctypes.byref(sz)) == 2
    assert lib.hyde_gram_workspace_size(164, 4096, 1, ctypes.byref(sz)) == 2
    assert lib.hyde_gram_workspace_size(32, 0, 1, ctypes.byref(sz)) == 2
    # allocation-free Gram: null pointers; its scratch size is a constant
    assert lib.hyde_gram_noalloc(None, 32, 4096, None, None) == 1
    assert lib.hyde_gram_noalloc_scratch_bytes() == 16 * 1024 * 1024
    # noise workspace: no output, one band, fewer pixels than bands
    assert lib.hyde_noise_est_workspace_size(32, 64, 64, None) == 1
    assert lib.hyde_noise_est_workspace_size(1, 64, 64, ctypes.byref(sz)) == 2
    assert lib.hyde_noise_est_workspace_size(32, 4, 4, ctypes.byref(sz)) == 2
    # layout query: no output, bad params
    lay = HydeWsLayout()
    assert lib.hyde_workspace_layout(32, 64, 64, ctypes.byref(prm), None) == 1
    bad = api.params(2, 8, 64)
    bad.wavelet = 4
    assert lib.hyde_workspace_layout(32, 64, 64, ctypes.byref(bad), ctypes.byref(lay)) == 1
    # timed entry point without its events
    assert lib.hyde_hyres_denoise_timed(1, 2, 32, 64, 64, ctypes.byref(prm), None, 3, 1 << 20,
                                        None, None) == 1
    # host cube stream: no cubes, missing device buffers or events
    ptrs4 = (ctypes.c_void_p * 4)(1, 2, 3, 4)
    evs7 = (ctypes.c_void_p * 7)(*range(1, 8))
    ys = (ctypes.c_void_p * 1)(5)
    xs = (ctypes.c_void_p * 1)(6)
    args = (ys, xs, None)
    tail = (32, 64, 64, ctypes.byref(prm))
    assert lib.hyde_hyres_denoise_host(*args, 0, *tail, ptrs4, 7, 8, 1 << 20, None, None,
                                       None, evs7) == 1
    holes = (ctypes.c_void_p * 4)(1, 2, None, 4)
    assert lib.hyde_hyres_denoise_host(*args, 1, *tail, holes, 7, 8, 1 << 20, None, None,
                                       None, evs7) == 1
    ev_holes = (ctypes.c_void_p * 7)(1, 2, 3, None, 5, 6, 7)
    assert lib.hyde_hyres_denoise_host(*args, 1, *tail, ptrs4, 7, 8, 1 << 20, None, None,
                                       None, ev_holes) == 1
    # windows: none, one outside the scene, a core outside its window
    ok = HydeWindow(0, 0, 32, 32, 8, 8, 16, 16)
    out = HydeWindow(40, 0, 32, 32, 48, 8, 16, 16)
    core = HydeWindow(0, 0, 32, 32, 24, 8, 16, 16)
    one = lambda w: (HydeWindow * 1)(w)
    assert lib.hyde_windows_workspace_size(8, 64, 64, one(ok), 0, ctypes.byref(prm), 4,
                                           ctypes.byref(sz)) == 1
    assert lib.hyde_windows_workspace_size(8, 64, 64, one(out), 1, ctypes.byref(prm), 4,
                                           ctypes.byref(sz)) == 2
    assert lib.hyde_windows_workspace_size(8, 64, 64, one(core), 1, ctypes.byref(prm), 4,
                                           ctypes.byref(sz)) == 2
    streams = (ctypes.c_void_p * 1)(9)
    assert lib.hyde_hyres_denoise_windows(1, 1, 8, 64, 64, one(ok), 1, ctypes.byref(prm), None,
                                          3, 1 << 20, streams, 1, evs7, None) == 1
    assert lib.hyde_hyres_denoise_windows(1, 2, 8, 64, 64, one(ok), 1, ctypes.byref(prm), None,
                                          3, 1 << 20, None, 1, evs7, None) == 1
    # backward: unknown loss, the MSE loss without its adjoint input
    assert lib.hyde_hyres_backward(1, 2, 32, 64, 64, ctypes.byref(prm), 3, 2, 4, None, 5,
                                   1 << 20, 6, 1 << 20, None) == 1
    assert lib.hyde_hyres_backward(1, None, 32, 64, 64, ctypes.byref(prm), 3, 0, 4, None, 5,
                                   1 << 20, 6, 1 << 20, None) == 1


@pytest.mark.parametrize("p,H,W,levels,r_max,K,code", [
    (32, 0, 64, 2, 8, 64, 2),      # empty image
    (32, 64, -1, 2, 8, 64, 2),     # negative side
    (1, 64, 64, 2, 1, 64, 2),      # one band: nothing to regress on
    (257, 64, 64, 2, 8, 64, 2),    # more bands than the Gram kernel takes
    (32, 64, 64, 2, 0, 64, 2),     # rank 0
    (32, 64, 64, 2, 33, 64, 2),    # rank above one warp per eigenpair
    (8, 64, 64, 2, 9, 64, 2),      # rank above the band count
    (32, 64, 64, 2, 8, 257, 2),    # more threshold candidates than the table holds
    (32, 64, 64, 0, 8, 64, 2),     # no DWT level
    (32, 64, 64, 11, 8, 64, 2),    # more levels than supported
    (32, 3, 64, 3, 8, 64, 2),      # padding (3 -> 8) longer than the image allows
    (32, 4, 4, 1, 8, 64, 2),       # fewer pixels than bands
])
def test_degenerate_shapes_rejected_on_host(lib, p, H, W, levels, r_max, K, code):
    from paper_2204_06979_gb300 import api
    sz = ctypes.c_size_t()
    prm = api.params(levels, r_max, K)
    assert lib.hyde_workspace_size(p, H, W, ctypes.byref(prm), ctypes.byref(sz)) == code


def test_hysime_rejects_bad_arguments_on_host(lib):
    """HySime's shape and pointer checks come before any device query."""
    sz = ctypes.c_size_t()
    assert lib.hyde_hysime_workspace_size(32, 4096, 8, None) == 1
    assert lib.hyde_hysime_workspace_size(1, 4096, 1, ctypes.byref(sz)) == 2      # one band
    assert lib.hyde_hysime_workspace_size(257, 4096, 8, ctypes.byref(sz)) == 2    # too many
    assert lib.hyde_hysime_workspace_size(32, 16, 8, ctypes.byref(sz)) == 2       # n < p
    assert lib.hyde_hysime_workspace_size(32, 4096, 0, ctypes.byref(sz)) == 2     # no candidate
    assert lib.hyde_hysime_workspace_size(32, 4096, 33, ctypes.byref(sz)) == 2    # above 32
    assert lib.hyde_hysime_workspace_size(8, 4096, 9, ctypes.byref(sz)) == 2      # above p
    assert lib.hyde_hysime(None, 32, 4096, 8, 1, 2, 3, 4, 5, None, 6, 1 << 20, None) == 1
    assert lib.hyde_hysime(1, 32, 4096, 8, 1, None, 3, 4, 5, None, 6, 1 << 20, None) == 1
    assert lib.hyde_hysime(1, 32, 16, 8, 1, 2, 3, 4, 5, None, 6, 1 << 20, None) == 2


def test_wait_limit_setter_round_trip(lib):
    """hyde_set_wait_limit_ns returns the previous limit; 0 is the default
    (one second)."""
    prev = lib.hyde_set_wait_limit_ns(1234)
    assert prev == 0
    assert lib.hyde_set_wait_limit_ns(0) == 1234
    assert lib.hyde_set_wait_limit_ns(0) == 0


def test_hyminor_rejects_bad_arguments_on_host(lib):
    """hyde_hyminor refuses null pointers, a negative lambda, a non-positive
    mu and an iteration count outside 1..100000 before touching the device."""
    from paper_2204_06979_gb300 import api
    prm = api.params(2, 8, 64)
    P = ctypes.byref(prm)
    assert lib.hyde_hyminor(None, 1, 8, 64, 64, P, 1.0, 10.0, 50, None, None, 0, None) == 1
    assert lib.hyde_hyminor(1, 1, 8, 64, 64, None, 1.0, 10.0, 50, None, None, 0, None) == 1
    assert lib.hyde_hyminor(1, 1, 8, 64, 64, P, -1.0, 10.0, 50, None, None, 0, None) == 1
    assert lib.hyde_hyminor(1, 1, 8, 64, 64, P, 1.0, 0.0, 50, None, None, 0, None) == 1
    assert lib.hyde_hyminor(1, 1, 8, 64, 64, P, 1.0, float("nan"), 50, None, None, 0, None) == 1
    assert lib.hyde_hyminor(1, 1, 8, 64, 64, P, 1.0, 10.0, 0, None, None, 0, None) == 2
    assert lib.hyde_hyminor_workspace_size(8, 64, 64, P, None) == 1


def test_forpdn_rejects_bad_shapes_on_host(lib):
    """hyde_forpdn_workspace_size checks its shape arguments on the host."""
    sz = ctypes.c_size_t()
    lib.hyde_forpdn_workspace_size.argtypes = [ctypes.c_int] * 5 + [ctypes.POINTER(ctypes.c_size_t)]
    assert lib.hyde_forpdn_workspace_size(8, 64, 64, 2, 64, None) == 1     # no output pointer
    assert lib.hyde_forpdn_workspace_size(1, 64, 64, 2, 64, ctypes.byref(sz)) == 2    # one band
    assert lib.hyde_forpdn_workspace_size(300, 64, 64, 2, 64, ctypes.byref(sz)) == 2  # p > 256
    assert lib.hyde_forpdn_workspace_size(8, 64, 64, 0, 64, ctypes.byref(sz)) == 2    # no level
    assert lib.hyde_forpdn_workspace_size(8, 64, 64, 2, 1, ctypes.byref(sz)) == 2     # K < 2
    assert lib.hyde_forpdn_workspace_size(8, 64, 64, 2, 300, ctypes.byref(sz)) == 2   # K > 256
    assert lib.hyde_forpdn_workspace_size(8, 2, 2, 1, 64, ctypes.byref(sz)) == 2      # n < p


def test_windows_plan_rejects_bad_tables_on_host(lib):
    """hyde_windows_plan_create checks the parameters and every window on the
    host before it asks for the device."""
    from paper_2204_06979_gb300 import api
    from paper_2204_06979_gb300._lib import HydeWindow
    plan = ctypes.c_void_p()

    def create(p, H, W, rows, prm):
        win = (HydeWindow * len(rows))(*[HydeWindow(*r) for r in rows])
        return lib.hyde_windows_plan_create(p, H, W, win, len(rows), ctypes.byref(prm),
                                            ctypes.byref(plan))

    ok_row = (0, 0, 64, 64, 0, 0, 64, 64)
    shared = api.params(2, 4, 64)
    assert lib.hyde_windows_plan_create(8, 64, 64, None, 1, ctypes.byref(shared),
                                        ctypes.byref(plan)) == 1
    assert create(8, 64, 64, [ok_row], api.params(2, 4, 64, lambda_mode=api.LAMBDA_PER_LEVEL)) == 1
    assert create(8, 64, 64, [ok_row], api.params(2, 4, 64, threshold_ll=True)) == 1
    assert create(8, 64, 64, [ok_row], api.params(2, 4, 64, precision=api.PREC_BF16X3)) == 1
    assert create(8, 64, 64, [ok_row], api.params(2, 4, 1)) == 1            # K < 2
    assert create(240, 64, 64, [ok_row], api.params(2, 4, 64)) == 2         # p > 208
    assert create(8, 64, 62, [(0, 0, 64, 62, 0, 0, 64, 62)], shared) == 2   # W not a multiple of 4
    assert create(8, 64, 64, [(0, 2, 64, 60, 0, 2, 64, 60)], shared) == 2   # x0 not a multiple of 4
    assert create(8, 64, 64, [(0, 0, 64, 68, 0, 0, 64, 64)], shared) == 2   # outside the scene
    assert create(8, 64, 64, [(0, 0, 32, 32, 0, 0, 40, 32)], shared) == 2   # core outside window
    assert create(8, 64, 64, [(0, 0, 3, 64, 0, 0, 3, 64)], api.params(3, 4, 64)) == 2  # padding
    assert plan.value is None
    assert lib.hyde_windows_plan_kernel_launches(None) == -1
    assert lib.hyde_windows_plan_destroy(None) == 1
    tile = ctypes.c_int()
    wgt = ctypes.c_double()
    assert lib.hyde_windows_plan_set_tuning(None, 256, 1.6) == 1
    assert lib.hyde_windows_plan_get_tuning(None, ctypes.byref(tile), ctypes.byref(wgt)) == 1
    assert lib.hyde_windows_plan_autotune(None, None, None, None, 0, None, None) == 1
