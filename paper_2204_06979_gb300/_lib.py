"""ctypes loader of libhyde.so and the C signatures of include/hyde.h.

The library must have been built (``python -m paper_2204_06979_gb300.build``
or ``__graft_entry__.build()``); a missing library raises immediately, there
is no fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libhyde.so")

c_int = ctypes.c_int
c_ll = ctypes.c_longlong
c_size = ctypes.c_size_t
c_vp = ctypes.c_void_p
c_size_p = ctypes.POINTER(ctypes.c_size_t)


class HydeParams(ctypes.Structure):
    _fields_ = [("wavelet", c_int), ("levels", c_int), ("r_max", c_int),
                ("n_lambda", c_int), ("precision", c_int), ("lambda_mode", c_int),
                ("threshold_ll", c_int), ("reserved", c_int)]


class HydeWindow(ctypes.Structure):
    _fields_ = [(name, c_int) for name in ("y0", "x0", "h", "w", "cy0", "cx0", "ch", "cw")]


class HydeWindowsWsLayout(ctypes.Structure):
    _fields_ = [(name, c_size) for name in ("R", "sigma", "V")]


class HydeWsLayout(ctypes.Structure):
    _fields_ = [(name, c_size) for name in
                ("total", "R", "sigma", "evals", "V", "coef", "sure", "sure_inf",
                 "sure_total", "status", "lam_comp")]


INFO_BYTES = 40   # hyde_hyres_info: 4 x int32 + 3 x float64
INFO_FORMAT = "<iiiiddd"

# name -> (restype, argtypes); every function declared in include/hyde.h
SIGNATURES = {
    "hyde_status_string": (ctypes.c_char_p, [c_int]),
    "hyde_version": (c_int, []),
    "hyde_gram_workspace_size": (c_int, [c_int, c_ll, c_int, c_size_p]),
    "hyde_gram": (c_int, [c_vp, c_int, c_ll, c_int, c_vp, c_vp, c_size, c_vp]),
    "hyde_gram_noalloc_scratch_bytes": (c_size, []),
    "hyde_gram_noalloc": (c_int, [c_vp, c_int, c_ll, c_vp, c_vp]),
    "hyde_noise_est_workspace_size": (c_int, [c_int, c_int, c_int, c_size_p]),
    "hyde_noise_est": (c_int, [c_vp, c_int, c_int, c_int, c_vp, c_vp, c_vp, c_size, c_vp]),
    "hyde_eig_workspace_size": (c_int, [c_int, c_int, c_size_p]),
    "hyde_eig_sym_top": (c_int, [c_vp, c_int, c_int, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "hyde_hysime_workspace_size": (c_int, [c_int, c_ll, c_int, c_size_p]),
    "hyde_hysime": (c_int, [c_vp, c_int, c_ll, c_int, c_vp, c_vp, c_vp, c_vp, c_vp, c_vp,
                            c_vp, c_size, c_vp]),
    "hyde_dwt_workspace_size": (c_int, [c_int, c_int, c_int, c_int, c_size_p]),
    "hyde_dwt2": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_int, c_vp, c_size, c_vp]),
    "hyde_idwt2": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_int, c_vp, c_size, c_vp]),
    "hyde_sure_workspace_size": (c_int, [c_int, c_int, c_size_p]),
    "hyde_sure_table": (c_int, [c_vp, c_int, c_int, c_int, c_int, c_int, c_vp, c_vp, c_vp,
                                c_size, c_vp]),
    "hyde_workspace_size": (c_int, [c_int, c_int, c_int, ctypes.POINTER(HydeParams), c_size_p]),
    "hyde_workspace_layout": (c_int, [c_int, c_int, c_int, ctypes.POINTER(HydeParams),
                                      ctypes.POINTER(HydeWsLayout)]),
    "hyde_hyres_denoise": (c_int, [c_vp, c_vp, c_int, c_int, c_int,
                                   ctypes.POINTER(HydeParams), c_vp, c_vp, c_size, c_vp]),
    "hyde_hyres_denoise_timed": (c_int, [c_vp, c_vp, c_int, c_int, c_int,
                                         ctypes.POINTER(HydeParams), c_vp, c_vp, c_size, c_vp,
                                         c_vp]),
    "hyde_hyres_kernel_launches": (c_int, [c_int, c_int, c_int, ctypes.POINTER(HydeParams)]),
    "hyde_set_grid_sm_cap": (c_int, [c_int]),
    "hyde_wsrrr_workspace_size": (c_int, [c_int, c_int, c_int, ctypes.POINTER(HydeParams),
                                          ctypes.POINTER(ctypes.c_size_t)]),
    "hyde_wsrrr": (c_int, [c_vp, c_vp, c_int, c_int, c_int, ctypes.POINTER(HydeParams), c_int,
                           c_vp, c_vp, c_vp, ctypes.c_size_t, c_vp]),
    "hyde_forpdn_workspace_size": (c_int, [c_int, c_int, c_int, c_int, c_int,
                                           ctypes.POINTER(ctypes.c_size_t)]),
    "hyde_forpdn": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int, c_int, c_vp, c_vp, c_vp,
                            ctypes.c_size_t, c_vp]),
    "hyde_hyminor_workspace_size": (c_int, [c_int, c_int, c_int, ctypes.POINTER(HydeParams),
                                            c_size_p]),
    "hyde_hyminor": (c_int, [c_vp, c_vp, c_int, c_int, c_int, ctypes.POINTER(HydeParams),
                             ctypes.c_float, ctypes.c_float, c_int, c_vp, c_vp, c_size, c_vp]),
    "hyde_set_wait_limit_ns": (ctypes.c_ulonglong, [ctypes.c_ulonglong]),
    "hyde_hyres_denoise_scaled": (c_int, [c_vp, c_vp, c_int, c_int, c_int,
                                          ctypes.POINTER(HydeParams), c_vp, c_vp, c_vp, c_size,
                                          c_vp]),
    "hyde_backward_workspace_size": (c_int, [c_int, c_int, c_int, ctypes.POINTER(HydeParams),
                                             c_size_p]),
    "hyde_hyres_backward": (c_int, [c_vp, c_vp, c_int, c_int, c_int, ctypes.POINTER(HydeParams),
                                    c_vp, c_int, c_vp, c_vp, c_vp, c_size, c_vp, c_size, c_vp]),
    "hyde_windows_workspace_size": (c_int, [c_int, c_int, c_int, c_vp, c_int,
                                            ctypes.POINTER(HydeParams), c_int, c_size_p]),
    "hyde_hyres_denoise_windows": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_vp, c_int,
                                           ctypes.POINTER(HydeParams), c_vp, c_vp, c_size, c_vp,
                                           c_int, c_vp, c_vp]),
    "hyde_windows_plan_create": (c_int, [c_int, c_int, c_int, c_vp, c_int,
                                         ctypes.POINTER(HydeParams), ctypes.POINTER(c_vp)]),
    "hyde_windows_plan_workspace_size": (c_int, [c_vp, c_size_p]),
    "hyde_windows_plan_kernel_launches": (c_int, [c_vp]),
    "hyde_windows_plan_destroy": (c_int, [c_vp]),
    "hyde_windows_plan_layout": (c_int, [c_vp, ctypes.POINTER(HydeWindowsWsLayout)]),
    "hyde_windows_plan_set_tuning": (c_int, [c_vp, c_int, ctypes.c_double]),
    "hyde_windows_plan_get_tuning": (c_int, [c_vp, ctypes.POINTER(c_int),
                                             ctypes.POINTER(ctypes.c_double)]),
    "hyde_windows_plan_autotune": (c_int, [c_vp, c_vp, c_vp, c_vp, c_size, c_vp,
                                           ctypes.POINTER(ctypes.c_float)]),
    "hyde_hyres_denoise_windows_batched": (c_int, [c_vp, c_vp, c_vp, c_vp, c_vp, c_size, c_vp]),
    "hyde_hyres_denoise_host": (c_int, [c_vp, c_vp, c_vp, c_int, c_int, c_int, c_int,
                                        ctypes.POINTER(HydeParams), c_vp, c_vp, c_vp, c_size,
                                        c_vp, c_vp, c_vp, c_vp]),
    "hyde_hyres_denoise_many": (c_int, [c_vp, c_vp, c_int, c_int, c_int, c_int,
                                        ctypes.POINTER(HydeParams), c_vp, c_vp, c_size, c_int,
                                        c_vp, c_vp, c_vp]),
}

N_STAGES = 8
STAGE_NAMES = ("gram", "noise", "eig", "project", "dwt", "sure", "idwt", "backproject")

_LIB = None


def load() -> ctypes.CDLL:
    """Load libhyde.so once and attach the C signatures."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(LIB_PATH):
        raise ImportError(
            f"{LIB_PATH} is missing: build it with `python -m paper_2204_06979_gb300.build` "
            "(nvcc with sm_103a); there is no CPU fallback")
    lib = ctypes.CDLL(LIB_PATH)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib
