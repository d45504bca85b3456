"""PyTorch-facing binding of libhyde (argument marshalling only).

Every function takes CUDA tensors, allocates outputs and workspaces with
torch's allocator, and calls the matching C entry point on the current torch
stream. All arithmetic runs in the library's CUDA kernels.
"""

from __future__ import annotations

import ctypes
import math
import struct

import torch

from . import _lib
from ._lib import HydeParams, HydeWsLayout, INFO_BYTES, INFO_FORMAT

HYDE_OK = 0
PREC_FP32 = 0
PREC_TF32X3 = 1       # Gram on the tensor cores (split-TF32, FP32-accurate)
PREC_BF16X3 = 2       # Gram on the tensor cores (split-BF16)
PREC_BF16X3_ALL = 3   # Gram, projection and back-projection on the tensor cores
LAMBDA_SHARED = 0         # one SURE threshold for every kept component
LAMBDA_PER_COMPONENT = 1  # each kept component at its own SURE threshold
LAMBDA_PER_LEVEL = 2      # each (kept component, level) at its own SURE threshold


class HydeError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.load().hyde_status_string(code).decode()
        super().__init__(f"{where}: {msg} (status {code})")
        self.code = code


def _check(code: int, where: str) -> None:
    if code != HYDE_OK:
        raise HydeError(code, where)


def _ptr(t: torch.Tensor | None) -> int | None:
    return None if t is None else t.data_ptr()


def _stream() -> int:
    return torch.cuda.current_stream().cuda_stream


def _cuda_f32(x: torch.Tensor, name: str) -> torch.Tensor:
    if not x.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if x.dtype != torch.float32:
        raise ValueError(f"{name} must be float32")
    return x.contiguous()


def _workspace(nbytes: int, device) -> torch.Tensor:
    # torch's caching allocator returns blocks aligned to at least 512 bytes
    return torch.empty(max(int(nbytes), 256), dtype=torch.uint8, device=device)


def padded_shape(H: int, W: int, levels: int) -> tuple[int, int]:
    q = 1 << levels
    return -(-H // q) * q, -(-W // q) * q


def params(levels: int, r_max: int, n_lambda: int = 64, precision: int = PREC_FP32,
           lambda_mode: int = LAMBDA_SHARED, threshold_ll: bool = False) -> HydeParams:
    p = HydeParams()
    p.wavelet = 2
    p.levels = levels
    p.r_max = r_max
    p.n_lambda = n_lambda
    p.precision = precision
    p.lambda_mode = lambda_mode
    p.threshold_ll = int(bool(threshold_ll))
    return p


def version() -> int:
    return _lib.load().hyde_version()


# ------------------------------------------------------------------ stages

def gram(Y: torch.Tensor, precision: int = PREC_FP32) -> torch.Tensor:
    """R = Y^T Y of a cube ``Y[p, ...]`` (float32, CUDA) as float64 ``[p, p]``
    (``precision`` PREC_FP32; PREC_TF32X3 or PREC_BF16X3 for the tensor-core
    forms)."""
    lib = _lib.load()
    Y = _cuda_f32(Y, "Y")
    p = Y.shape[0]
    n = Y.numel() // p
    sz = ctypes.c_size_t()
    _check(lib.hyde_gram_workspace_size(p, n, precision, ctypes.byref(sz)), "hyde_gram_workspace_size")
    ws = _workspace(sz.value, Y.device)
    R = torch.empty((p, p), dtype=torch.float64, device=Y.device)
    _check(lib.hyde_gram(_ptr(Y), p, n, precision, _ptr(R), _ptr(ws), ws.numel(), _stream()),
           "hyde_gram")
    return R


def noise_est(Y: torch.Tensor) -> tuple[torch.Tensor, torch.Tensor]:
    """Per-band noise std of ``Y[p, H, W]`` by multiple regression.
    Returns ``(sigma float64[p], status int32[1])``."""
    lib = _lib.load()
    Y = _cuda_f32(Y, "Y")
    p, H, W = Y.shape
    sz = ctypes.c_size_t()
    _check(lib.hyde_noise_est_workspace_size(p, H, W, ctypes.byref(sz)), "hyde_noise_est_workspace_size")
    ws = _workspace(sz.value, Y.device)
    sigma = torch.empty(p, dtype=torch.float64, device=Y.device)
    status = torch.zeros(1, dtype=torch.int32, device=Y.device)
    _check(lib.hyde_noise_est(_ptr(Y), p, H, W, _ptr(sigma), _ptr(status), _ptr(ws), ws.numel(),
                              _stream()), "hyde_noise_est")
    return sigma, status


def eig_sym_top(A: torch.Tensor, r: int) -> tuple[torch.Tensor, torch.Tensor, torch.Tensor]:
    """Leading r eigenpairs of a symmetric float64 CUDA matrix.
    Returns ``(evals[r], V[p, r], status[1])``."""
    lib = _lib.load()
    if not A.is_cuda or A.dtype != torch.float64:
        raise ValueError("A must be a float64 CUDA tensor")
    A = A.contiguous()
    p = A.shape[0]
    sz = ctypes.c_size_t()
    _check(lib.hyde_eig_workspace_size(p, r, ctypes.byref(sz)), "hyde_eig_workspace_size")
    ws = _workspace(sz.value, A.device)
    evals = torch.empty(r, dtype=torch.float64, device=A.device)
    V = torch.empty((p, r), dtype=torch.float64, device=A.device)
    status = torch.zeros(1, dtype=torch.int32, device=A.device)
    _check(lib.hyde_eig_sym_top(_ptr(A), p, r, _ptr(evals), _ptr(V), _ptr(status), _ptr(ws),
                                ws.numel(), _stream()), "hyde_eig_sym_top")
    return evals, V, status


def hysime(Y: torch.Tensor, r_max: int = 32) -> dict:
    """HySime subspace identification of ``Y`` (``[p, H, W]`` or ``[p, n]``,
    float32, CUDA) with the ``min(r_max, p, 32)`` leading eigenvectors of the
    signal correlation as candidates. Synchronises to read the dimension;
    returns ``k``, ``E`` (``p x k``, the kept eigenvectors in ascending
    delta), ``idx``, all candidates' ``V``, ``delta`` and ``evals``, and
    ``saturated`` (every candidate kept while there are fewer candidates
    than bands: ``k`` is then only a lower bound)."""
    Y = _cuda_f32(Y, "Y")
    lib = _lib.load()
    p = Y.shape[0]
    n = Y.numel() // p
    r = min(r_max, p, 32)
    sz = ctypes.c_size_t()
    _check(lib.hyde_hysime_workspace_size(p, n, r, ctypes.byref(sz)), "hyde_hysime_workspace_size")
    ws = _workspace(sz.value, Y.device)
    dev = Y.device
    k = torch.zeros(1, dtype=torch.int32, device=dev)
    idx = torch.empty(r, dtype=torch.int32, device=dev)
    V = torch.empty(p, r, dtype=torch.float64, device=dev)
    delta = torch.empty(r, dtype=torch.float64, device=dev)
    evals = torch.empty(r, dtype=torch.float64, device=dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    _check(lib.hyde_hysime(_ptr(Y), p, n, r, _ptr(k), _ptr(idx), _ptr(V), _ptr(delta),
                           _ptr(evals), _ptr(status), _ptr(ws), ws.numel(), _stream()),
           "hyde_hysime")
    kk = int(k.item())
    keep = idx[:kk].long()
    # every candidate kept with fewer candidates than bands: k is a lower bound
    saturated = kk == r and r < p
    return dict(k=kk, E=V[:, keep], idx=keep, V=V, delta=delta, evals=evals,
                status=int(status.item()), saturated=saturated)


def dwt2(x: torch.Tensor, levels: int) -> torch.Tensor:
    """Periodic db2 analysis of ``x[B, H, W]`` -> Mallat ``coef[B, Hp, Wp]``."""
    lib = _lib.load()
    x = _cuda_f32(x, "x")
    B, H, W = x.shape
    Hp, Wp = padded_shape(H, W, levels)
    sz = ctypes.c_size_t()
    _check(lib.hyde_dwt_workspace_size(B, H, W, levels, ctypes.byref(sz)), "hyde_dwt_workspace_size")
    ws = _workspace(sz.value, x.device)
    coef = torch.empty((B, Hp, Wp), dtype=torch.float32, device=x.device)
    _check(lib.hyde_dwt2(_ptr(x), _ptr(coef), B, H, W, 2, levels, _ptr(ws), ws.numel(), _stream()),
           "hyde_dwt2")
    return coef


def idwt2(coef: torch.Tensor, H: int, W: int, levels: int) -> torch.Tensor:
    """Inverse of ``dwt2``: ``coef[B, Hp, Wp]`` -> ``x[B, H, W]``."""
    lib = _lib.load()
    coef = _cuda_f32(coef, "coef")
    B = coef.shape[0]
    if tuple(coef.shape[1:]) != padded_shape(H, W, levels):
        raise ValueError("coef shape does not match (H, W, levels)")
    sz = ctypes.c_size_t()
    _check(lib.hyde_dwt_workspace_size(B, H, W, levels, ctypes.byref(sz)), "hyde_dwt_workspace_size")
    ws = _workspace(sz.value, coef.device)
    out = torch.empty((B, H, W), dtype=torch.float32, device=coef.device)
    _check(lib.hyde_idwt2(_ptr(coef), _ptr(out), B, H, W, 2, levels, _ptr(ws), ws.numel(),
                          _stream()), "hyde_idwt2")
    return out


def sure_table(coef: torch.Tensor, levels: int, K: int = 64) -> tuple[torch.Tensor, torch.Tensor]:
    """SURE of soft-thresholding each image of ``coef[B, Hp, Wp]`` on the
    K-point grid, and of dropping it: ``(S[B, K], S_inf[B])`` float64."""
    lib = _lib.load()
    coef = _cuda_f32(coef, "coef")
    B, Hp, Wp = coef.shape
    sz = ctypes.c_size_t()
    _check(lib.hyde_sure_workspace_size(B, K, ctypes.byref(sz)), "hyde_sure_workspace_size")
    ws = _workspace(sz.value, coef.device)
    S = torch.empty((B, K), dtype=torch.float64, device=coef.device)
    S_inf = torch.empty(B, dtype=torch.float64, device=coef.device)
    _check(lib.hyde_sure_table(_ptr(coef), B, Hp, Wp, levels, K, _ptr(S), _ptr(S_inf), _ptr(ws),
                               ws.numel(), _stream()), "hyde_sure_table")
    return S, S_inf


# ------------------------------------------------------------ whole path

def parse_info(info: torch.Tensor) -> dict:
    raw = bytes(info.cpu().numpy().tobytes())
    st, rank, k, _, lam, smin, gap = struct.unpack(INFO_FORMAT, raw[:INFO_BYTES])
    return dict(status=st, rank=rank, lambda_index=k, lam=lam, sure_min=smin, sure_gap=gap)


class HyRes:
    """Reusable HyRes denoiser for cubes of one shape: owns the workspace and
    the device info record; ``__call__`` enqueues one denoise on the current
    stream."""

    def __init__(self, p: int, H: int, W: int, levels: int, r_max: int, n_lambda: int = 64,
                 device="cuda", precision: int = PREC_FP32, lambda_mode: int = LAMBDA_SHARED,
                 threshold_ll: bool = False):
        self.lib = _lib.load()
        self.shape = (p, H, W)
        self.params = params(levels, r_max, n_lambda, precision, lambda_mode, threshold_ll)
        sz = ctypes.c_size_t()
        _check(self.lib.hyde_workspace_size(p, H, W, ctypes.byref(self.params), ctypes.byref(sz)),
               "hyde_workspace_size")
        self.layout = HydeWsLayout()
        _check(self.lib.hyde_workspace_layout(p, H, W, ctypes.byref(self.params),
                                              ctypes.byref(self.layout)), "hyde_workspace_layout")
        self.device = torch.device(device)
        self.ws = _workspace(sz.value, self.device)
        self.info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=self.device)

    def __call__(self, Y: torch.Tensor, X: torch.Tensor | None = None) -> torch.Tensor:
        Y = _cuda_f32(Y, "Y")
        if tuple(Y.shape) != self.shape:
            raise ValueError(f"expected a cube of shape {self.shape}")
        if X is None:
            X = torch.empty_like(Y)
        p, H, W = self.shape
        _check(self.lib.hyde_hyres_denoise(_ptr(Y), _ptr(X), p, H, W, ctypes.byref(self.params),
                                           _ptr(self.info), _ptr(self.ws), self.ws.numel(),
                                           _stream()), "hyde_hyres_denoise")
        return X

    def result_info(self) -> dict:
        return parse_info(self.info)

    def denoise_host(self, Ys, Xs, infos: torch.Tensor | None = None) -> None:
        """Denoises the host cubes ``Ys[s]`` into ``Xs[s]`` (contiguous float32
        CPU tensors of this shape, page-locked for the copies to overlap) with
        ``hyde_hyres_denoise_host``: cube s+1 is copied in and cube s-1 out
        while cube s is denoised. Enqueued on the current stream (synchronise
        before reading ``Xs``). ``infos``: optional page-locked uint8 tensor of
        ``len(Ys) * INFO_BYTES`` bytes for the per-cube records."""
        n = len(Ys)
        if n < 1 or len(Xs) != n:
            raise ValueError("Ys and Xs must be equally long and non-empty")
        for t in list(Ys) + list(Xs):
            if (t.device.type != "cpu" or t.dtype != torch.float32 or not t.is_contiguous()
                    or tuple(t.shape) != self.shape):
                raise ValueError(f"host cubes must be contiguous float32 CPU tensors of shape "
                                 f"{self.shape}")
        if infos is not None and (infos.device.type != "cpu" or infos.numel() < n * INFO_BYTES):
            raise ValueError("infos must be a CPU uint8 tensor of len(Ys) * INFO_BYTES bytes")
        if not hasattr(self, "_host_dev"):
            self._host_bufs = [torch.empty(self.shape, dtype=torch.float32, device=self.device)
                               for _ in range(4)]
            self._host_info = torch.zeros(2 * INFO_BYTES, dtype=torch.uint8, device=self.device)
            self._host_streams = [torch.cuda.Stream(device=self.device) for _ in range(2)]
            self._host_events = [torch.cuda.Event() for _ in range(7)]
            for e in self._host_events:   # torch creates the CUDA event on first record
                e.record(torch.cuda.current_stream(self.device))
            torch.cuda.synchronize(self.device)
            self._host_dev = (ctypes.c_void_p * 4)(*[t.data_ptr() for t in self._host_bufs])
            self._host_ev = (ctypes.c_void_p * 7)(*[e.cuda_event for e in self._host_events])
        Yp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Ys])
        Xp = (ctypes.c_void_p * n)(*[t.data_ptr() for t in Xs])
        p, H, W = self.shape
        _check(self.lib.hyde_hyres_denoise_host(
            Yp, Xp, _ptr(infos), n, p, H, W, ctypes.byref(self.params), self._host_dev,
            _ptr(self._host_info), _ptr(self.ws), self.ws.numel(), _stream(),
            self._host_streams[0].cuda_stream, self._host_streams[1].cuda_stream,
            self._host_ev), "hyde_hyres_denoise_host")

    def _view(self, off: int, count: int, dtype: torch.dtype) -> torch.Tensor:
        es = torch.tensor([], dtype=dtype).element_size()
        return self.ws[off: off + count * es].view(dtype)

    def intermediates(self) -> dict:
        """Views into the workspace of the last call's intermediates."""
        p, H, W = self.shape
        r, K = self.params.r_max, self.params.n_lambda
        Hp, Wp = padded_shape(H, W, self.params.levels)
        L = self.layout
        lv = self.params.levels
        # per-level mode: one SURE row per (component, level)
        s_shape = (r, lv, K) if self.params.lambda_mode == LAMBDA_PER_LEVEL else (r, K)
        return dict(
            R=self._view(L.R, p * p, torch.float64).view(p, p),
            sigma=self._view(L.sigma, p, torch.float64),
            evals=self._view(L.evals, r, torch.float64),
            V=self._view(L.V, p * r, torch.float64).view(p, r),
            coef=self._view(L.coef, r * Hp * Wp, torch.float32).view(r, Hp, Wp),
            S=self._view(L.sure, math.prod(s_shape), torch.float64).view(*s_shape),
            S_inf=self._view(L.sure_inf, r, torch.float64),
            T=self._view(L.sure_total, r * K, torch.float64).view(r, K),
            status=self._view(L.status, 1, torch.int32),
            lam_comp=self._view(L.lam_comp, r * self.params.levels,
                                torch.float32).view(r, self.params.levels),
        )


class HyResMany:
    """Several cubes of one shape at once (``hyde_hyres_denoise_many``): ``slots``
    workspaces, each with its own stream, forked from and joined to the
    current stream; cube k runs in slot k % slots, so one cube's
    single-block stages overlap another's bandwidth-bound ones (four slots
    measured fastest of one to four on a 349 x 1905 x 144 cube)."""

    def __init__(self, p: int, H: int, W: int, levels: int, r_max: int, n_lambda: int = 64,
                 slots: int = 4, device="cuda", precision: int = PREC_FP32):
        self.lib = _lib.load()
        self.shape = (p, H, W)
        self.params = params(levels, r_max, n_lambda, precision)
        sz = ctypes.c_size_t()
        _check(self.lib.hyde_workspace_size(p, H, W, ctypes.byref(self.params), ctypes.byref(sz)),
               "hyde_workspace_size")
        self.device = torch.device(device)
        self.slots = int(slots)
        self.ws = [_workspace(sz.value, self.device) for _ in range(self.slots)]
        self.ws_bytes = sz.value
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.slots)]
        self.events = [torch.cuda.Event() for _ in range(self.slots + 1)]
        cur = torch.cuda.current_stream(self.device)
        for e in self.events:   # torch creates the CUDA event on first record
            e.record(cur)
        self.info = None

    def __call__(self, Ys, Xs) -> None:
        """Enqueues ``Ys[k] -> Xs[k]`` for every k on the current stream's
        timeline (returns at once)."""
        count = len(Ys)
        if count != len(Xs) or count < 1:
            raise ValueError("need as many outputs as inputs")
        for Y, X in zip(Ys, Xs):
            if tuple(Y.shape) != self.shape or tuple(X.shape) != self.shape:
                raise ValueError("every cube must have the shape the plan was made for")
            _cuda_f32(Y, "Y")
            _cuda_f32(X, "X")
        if self.info is None or self.info.numel() != count * INFO_BYTES:
            self.info = torch.zeros(count * INFO_BYTES, dtype=torch.uint8, device=self.device)
        p, H, W = self.shape
        yp = (ctypes.c_void_p * count)(*[Y.data_ptr() for Y in Ys])
        xp = (ctypes.c_void_p * count)(*[X.data_ptr() for X in Xs])
        wp = (ctypes.c_void_p * self.slots)(*[w.data_ptr() for w in self.ws])
        sp = (ctypes.c_void_p * self.slots)(*[s.cuda_stream for s in self.streams])
        ep = (ctypes.c_void_p * (self.slots + 1))(*[e.cuda_event for e in self.events])
        _check(self.lib.hyde_hyres_denoise_many(yp, xp, count, p, H, W, ctypes.byref(self.params),
                                                self.info.data_ptr(), wp, self.ws_bytes,
                                                self.slots, _stream(), sp, ep),
               "hyde_hyres_denoise_many")

    def result_info(self, k: int) -> dict:
        """The info record of cube k of the last call (synchronises)."""
        torch.cuda.current_stream(self.device).synchronize()
        return parse_info(self.info[k * INFO_BYTES:(k + 1) * INFO_BYTES])


def hyres_denoise(Y: torch.Tensor, levels: int, r_max: int, n_lambda: int = 64,
                  precision: int = PREC_FP32, lambda_mode: int = LAMBDA_SHARED,
                  threshold_ll: bool = False):
    """One-shot HyRes on ``Y[p, H, W]``; returns ``(X, info dict)``
    (synchronises the current stream to read the info record)."""
    p, H, W = Y.shape
    h = HyRes(p, H, W, levels, r_max, n_lambda, device=Y.device, precision=precision,
              lambda_mode=lambda_mode, threshold_ll=threshold_ll)
    X = h(Y)
    return X, h.result_info()


# ------------------------------------------------------ differentiation form

def hyminor(Y: torch.Tensor, levels: int, r_max: int, n_lambda: int = 64, lam: float = 1.0,
            mu: float = 10.0, iters: int = 50, precision: int = PREC_FP32
            ) -> tuple[torch.Tensor, dict]:
    """HyMiNoR of ``Y[p, H, W]`` (``hyde_hyminor``): HyRes, then the l1-l1
    sparse-noise stage. Returns ``(X, info)`` (info: HyRes's choice)."""
    lib = _lib.load()
    Y = _cuda_f32(Y, "Y")
    p, H, W = Y.shape
    prm = params(levels, r_max, n_lambda, precision)
    sz = ctypes.c_size_t()
    _check(lib.hyde_hyminor_workspace_size(p, H, W, ctypes.byref(prm), ctypes.byref(sz)),
           "hyde_hyminor_workspace_size")
    ws = _workspace(sz.value, Y.device)
    X = torch.empty_like(Y)
    info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=Y.device)
    _check(lib.hyde_hyminor(_ptr(Y), _ptr(X), p, H, W, ctypes.byref(prm), float(lam), float(mu),
                            int(iters), _ptr(info), _ptr(ws), ws.numel(), _stream()),
           "hyde_hyminor")
    return X, parse_info(info)


def wsrrr(Y: torch.Tensor, levels: int, r_max: int, n_lambda: int = 64, iters: int = 10,
          precision: int = PREC_FP32, features: bool = False
          ) -> tuple[torch.Tensor, dict] | tuple[torch.Tensor, dict, torch.Tensor]:
    """WSRRR of ``Y[p, H, W]`` (``hyde_wsrrr``): HyRes, then ``iters`` cyclic
    descent steps on the sparse reduced-rank model. Returns ``(X, info)``
    (info: HyRes's choice), and with ``features`` also the component images
    ``F[r_max, H_p, W_p]`` (rows past the rank zero)."""
    lib = _lib.load()
    Y = _cuda_f32(Y, "Y")
    p, H, W = Y.shape
    prm = params(levels, r_max, n_lambda, precision)
    sz = ctypes.c_size_t()
    _check(lib.hyde_wsrrr_workspace_size(p, H, W, ctypes.byref(prm), ctypes.byref(sz)),
           "hyde_wsrrr_workspace_size")
    ws = _workspace(sz.value, Y.device)
    X = torch.empty_like(Y)
    info = torch.zeros(INFO_BYTES, dtype=torch.uint8, device=Y.device)
    F = None
    if features:
        Hp, Wp = padded_shape(H, W, levels)
        F = torch.empty((r_max, Hp, Wp), dtype=torch.float32, device=Y.device)
    _check(lib.hyde_wsrrr(_ptr(Y), _ptr(X), p, H, W, ctypes.byref(prm), int(iters), _ptr(info),
                          _ptr(F), _ptr(ws), ws.numel(), _stream()), "hyde_wsrrr")
    if features:
        return X, parse_info(info), F
    return X, parse_info(info)


def forpdn(Y: torch.Tensor, levels: int, n_lambda: int = 64) -> tuple[torch.Tensor, dict]:
    """FORPDN of ``Y[p, H, W]`` (``hyde_forpdn``): per wavelet-level group,
    spectral smoothing (I + lam D^T D)^-1 with lam chosen by SURE. Returns
    ``(X, info)`` with info's ``status``, the chosen grid index per group
    (``k``, group 0 = the final LL band) and the SURE table (``sure``)."""
    lib = _lib.load()
    Y = _cuda_f32(Y, "Y")
    p, H, W = Y.shape
    sz = ctypes.c_size_t()
    _check(lib.hyde_forpdn_workspace_size(p, H, W, levels, n_lambda, ctypes.byref(sz)),
           "hyde_forpdn_workspace_size")
    ws = _workspace(sz.value, Y.device)
    X = torch.empty_like(Y)
    info = torch.zeros(levels + 2, dtype=torch.int32, device=Y.device)
    sure = torch.zeros((levels + 1, n_lambda), dtype=torch.float64, device=Y.device)
    _check(lib.hyde_forpdn(_ptr(Y), _ptr(X), p, H, W, levels, n_lambda, _ptr(info), _ptr(sure),
                           _ptr(ws), ws.numel(), _stream()), "hyde_forpdn")
    inf = info.cpu().tolist()
    return X, {"status": inf[0], "k": inf[1:], "sure": sure}


def _scale_rows(scale: torch.Tensor, r_max: int, levels: int) -> torch.Tensor:
    if not scale.is_cuda or scale.dtype != torch.float32 or scale.dim() != 2:
        raise ValueError("scale must be a float32 CUDA matrix [rows >= r_max, levels]")
    if scale.shape[0] < r_max or scale.shape[1] != levels:
        raise ValueError(f"scale must have >= {r_max} rows and {levels} columns")
    return scale[:r_max].contiguous()


class HyResGrad(HyRes):
    """HyRes with per-(component, level) threshold scales and the hand-written
    backward. Owns a forward workspace (which the backward reads) and a
    backward workspace; use one instance per cube of a batch."""

    def __init__(self, p, H, W, levels, r_max, n_lambda=64, device="cuda"):
        super().__init__(p, H, W, levels, r_max, n_lambda, device)
        sz = ctypes.c_size_t()
        _check(self.lib.hyde_backward_workspace_size(p, H, W, ctypes.byref(self.params),
                                                     ctypes.byref(sz)),
               "hyde_backward_workspace_size")
        self.bws = _workspace(sz.value, self.device)
        self.sure_value = torch.zeros(1, dtype=torch.float64, device=self.device)

    def forward_scaled(self, Y: torch.Tensor, scale: torch.Tensor) -> torch.Tensor:
        Y = _cuda_f32(Y, "Y")
        s = _scale_rows(scale, self.params.r_max, self.params.levels)
        X = torch.empty_like(Y)
        p, H, W = self.shape
        _check(self.lib.hyde_hyres_denoise_scaled(
            _ptr(Y), _ptr(X), p, H, W, ctypes.byref(self.params), _ptr(s), _ptr(self.info),
            _ptr(self.ws), self.ws.numel(), _stream()), "hyde_hyres_denoise_scaled")
        return X

    def backward_scaled(self, Y: torch.Tensor, dX: torch.Tensor | None, scale: torch.Tensor,
                        loss: int = 0) -> torch.Tensor:
        """dL/dscale as float32 [r_max, levels] (loss 0: dX = dL/dX_hat;
        loss 1: the SURE loss, value left in ``self.sure_value``)."""
        Y = _cuda_f32(Y, "Y")
        s = _scale_rows(scale, self.params.r_max, self.params.levels)
        ds = torch.empty((self.params.r_max, self.params.levels), dtype=torch.float32,
                         device=self.device)
        p, H, W = self.shape
        dptr = None
        if loss == 0:
            dX = _cuda_f32(dX, "dX")
            dptr = _ptr(dX)
        _check(self.lib.hyde_hyres_backward(
            _ptr(Y), dptr, p, H, W, ctypes.byref(self.params), _ptr(s), loss, _ptr(ds),
            _ptr(self.sure_value), _ptr(self.ws), self.ws.numel(), _ptr(self.bws),
            self.bws.numel(), _stream()), "hyde_hyres_backward")
        return ds


def _pad_rows(ds: torch.Tensor, like: torch.Tensor) -> torch.Tensor:
    out = torch.zeros_like(like)
    out[: ds.shape[0]] = ds
    return out


class HyResScaledFn(torch.autograd.Function):
    """X_hat = HyRes_s(Y): differentiable in the threshold scales only (the
    cube is data; the rank and base threshold are stop-gradient)."""

    @staticmethod
    def forward(ctx, Y, scale, model):
        X = model.forward_scaled(Y, scale)
        ctx.model = model
        ctx.save_for_backward(Y, scale)
        return X

    @staticmethod
    def backward(ctx, gX):
        Y, scale = ctx.saved_tensors
        ds = ctx.model.backward_scaled(Y, gX.contiguous(), scale, loss=0)
        return None, _pad_rows(ds, scale), None


class HyResSureFn(torch.autograd.Function):
    """SURE of the kept components with thresholds lambda* scale (a scalar,
    float64), with its almost-everywhere gradient in the scales."""

    @staticmethod
    def forward(ctx, Y, scale, model):
        model.forward_scaled(Y, scale)            # rank, lambda* and weights
        ds = model.backward_scaled(Y, None, scale, loss=1)
        ctx.save_for_backward(_pad_rows(ds, scale))
        return model.sure_value.clone().reshape(())

    @staticmethod
    def backward(ctx, g):
        (ds,) = ctx.saved_tensors
        return None, ds * g.to(ds.dtype), None


class _GridSmCap:
    """Caps the SM count the library sizes grids from, for launches made by
    this host thread inside the ``with`` block (``hyde_set_grid_sm_cap``)."""

    def __init__(self, sms: int):
        self.sms = int(sms)

    def __enter__(self):
        self.prev = _lib.load().hyde_set_grid_sm_cap(self.sms) if self.sms > 0 else None
        return self

    def __exit__(self, *exc):
        if self.prev is not None:
            _lib.load().hyde_set_grid_sm_cap(self.prev)
        return False


class HyResScaledBatchFn(torch.autograd.Function):
    """A batch of cubes through the scaled HyRes with shared threshold scales:
    each cube's forward and backward run on their own stream, forked from
    the caller's stream and joined back to it, so the cubes' pipelines (each
    latency-bound on a few SMs) overlap on the GPU. dL/dscale is the sum over
    the cubes."""

    @staticmethod
    def forward(ctx, scale, models, streams, sm_cap, *Ys):
        cur = torch.cuda.current_stream(scale.device)
        outs = []
        with _GridSmCap(sm_cap):
            for Y, m, st in zip(Ys, models, streams):
                st.wait_stream(cur)
                Y.record_stream(st)
                scale.record_stream(st)
                with torch.cuda.stream(st):
                    outs.append(m.forward_scaled(Y, scale))
        for X, st in zip(outs, streams):
            cur.wait_stream(st)
            X.record_stream(cur)
        ctx.models, ctx.streams, ctx.sm_cap = models, streams, sm_cap
        ctx.save_for_backward(scale, *Ys)
        return tuple(outs)

    @staticmethod
    def backward(ctx, *gXs):
        scale, *Ys = ctx.saved_tensors
        cur = torch.cuda.current_stream(scale.device)
        dss = []
        with _GridSmCap(ctx.sm_cap):
            for Y, g, m, st in zip(Ys, gXs, ctx.models, ctx.streams):
                st.wait_stream(cur)
                g = g.contiguous()
                g.record_stream(st)
                Y.record_stream(st)
                with torch.cuda.stream(st):
                    dss.append(m.backward_scaled(Y, g, scale, loss=0))
        total = torch.zeros_like(scale)
        for ds, st in zip(dss, ctx.streams):
            cur.wait_stream(st)
            ds.record_stream(cur)
            total[: ds.shape[0]] += ds
        return (total, None, None, None) + (None,) * len(Ys)


def hyres_scaled(Y: torch.Tensor, scale: torch.Tensor, model: HyResGrad) -> torch.Tensor:
    return HyResScaledFn.apply(Y, scale, model)


def hyres_scaled_batch(Ys, scale: torch.Tensor, models, streams=None, sm_cap: int | None = None):
    """``[HyRes_s(Y) for Y in Ys]`` with each cube on its own stream (one
    HyResGrad per cube; ``streams`` default to new ones). ``sm_cap`` > 0 sizes
    the library's grids for that many SMs (``hyde_set_grid_sm_cap``), 0 for
    all of them; by default an eighth of the SMs when four or more cubes run
    concurrently, so that each cube's multi-block kernels leave SMs free for
    the others' one-block kernels (16 cubes of 128 x 128 x 64: 1.03 ms per
    training step uncapped, 0.95 at 9 SMs, 0.93 at 19, 0.95 at 38)."""
    if len(Ys) != len(models):
        raise ValueError("one model per cube")
    if streams is None:
        streams = [torch.cuda.Stream(scale.device) for _ in Ys]
    if sm_cap is None:
        sms = torch.cuda.get_device_properties(scale.device).multi_processor_count
        sm_cap = max(1, sms // 8) if len(Ys) >= 4 else 0
    return list(HyResScaledBatchFn.apply(scale, list(models), list(streams), int(sm_cap), *Ys))


def hyres_sure_loss(Y: torch.Tensor, scale: torch.Tensor, model: HyResGrad) -> torch.Tensor:
    return HyResSureFn.apply(Y, scale, model)


# ------------------------------------------------------- sliding windows

class HyResWindowsBatched:
    """Sliding-window HyRes with one launch per stage over all windows
    (``hyde_hyres_denoise_windows_batched``): a plan built once from the
    window table (``int32[n][8]``, as for ``HyResWindows``), its workspace and
    per-window info records. ``__call__`` enqueues the scene on the current
    stream; ``capture``/``replay`` record it into a CUDA graph."""

    def __init__(self, p, H, W, table, levels, r_max, n_lambda=64, device="cuda",
                 precision: int = PREC_FP32):
        from ._lib import HydeWindow
        self.lib = _lib.load()
        self.shape = (p, H, W)
        self.params = params(levels, r_max, n_lambda, precision=precision)
        self.device = torch.device(device)
        rows = [tuple(int(v) for v in r) for r in table]
        self.n_win = len(rows)
        win = (HydeWindow * self.n_win)(*[HydeWindow(*r) for r in rows])
        self._table = win
        self.plan = ctypes.c_void_p()
        _check(self.lib.hyde_windows_plan_create(p, H, W, win, self.n_win,
                                                 ctypes.byref(self.params),
                                                 ctypes.byref(self.plan)),
               "hyde_windows_plan_create")
        sz = ctypes.c_size_t()
        _check(self.lib.hyde_windows_plan_workspace_size(self.plan, ctypes.byref(sz)),
               "hyde_windows_plan_workspace_size")
        self.ws = _workspace(sz.value, self.device)
        self.info = torch.zeros(self.n_win * INFO_BYTES, dtype=torch.uint8, device=self.device)
        self.kernel_launches = self.lib.hyde_windows_plan_kernel_launches(self.plan)
        self.graph = None

    def __del__(self):
        plan = getattr(self, "plan", None)
        if plan is not None and plan.value:
            self.lib.hyde_windows_plan_destroy(plan)
            self.plan = None

    def __call__(self, Y: torch.Tensor, X: torch.Tensor | None = None) -> torch.Tensor:
        Y = _cuda_f32(Y, "Y")
        if tuple(Y.shape) != self.shape:
            raise ValueError(f"expected a scene of shape {self.shape}")
        if X is None:
            X = torch.empty_like(Y)
        _check(self.lib.hyde_hyres_denoise_windows_batched(
            _ptr(Y), _ptr(X), self.plan, _ptr(self.info), _ptr(self.ws), self.ws.numel(),
            _stream()), "hyde_hyres_denoise_windows_batched")
        return X

    def capture(self, Y: torch.Tensor, X: torch.Tensor) -> None:
        """Record one scene denoise (reading Y, writing X) into a CUDA graph."""
        self(Y, X)
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self(Y, X)

    def replay(self) -> None:
        self.graph.replay()

    def infos(self) -> list[dict]:
        raw = self.info.cpu()
        return [parse_info(raw[k * INFO_BYTES:(k + 1) * INFO_BYTES]) for k in range(self.n_win)]

    def tuning(self) -> dict:
        """The plan's tuned settings: projection tile and Gram role weight."""
        tile = ctypes.c_int()
        w = ctypes.c_double()
        _check(self.lib.hyde_windows_plan_get_tuning(self.plan, ctypes.byref(tile),
                                                     ctypes.byref(w)),
               "hyde_windows_plan_get_tuning")
        return {"proj_tile": tile.value, "gram_role_weight": w.value}

    def set_tuning(self, proj_tile: int, gram_role_weight: float) -> None:
        _check(self.lib.hyde_windows_plan_set_tuning(self.plan, int(proj_tile),
                                                     float(gram_role_weight)),
               "hyde_windows_plan_set_tuning")
        self.graph = None   # a captured call keeps the grid sizes it was captured with

    def _cache_key(self) -> str:
        import hashlib
        h = hashlib.sha1()
        h.update(repr((self.shape, self.params.levels, self.params.r_max,
                       self.params.n_lambda, torch.cuda.get_device_name(self.device))).encode())
        h.update(bytes(self._table))
        return h.hexdigest()

    def autotune(self, Y: torch.Tensor, X: torch.Tensor | None = None,
                 cache: str | None = None) -> dict:
        """Pick the fastest tuning on this scene (hyde_windows_plan_autotune)
        and return it with its time. With a cache file (JSON), a setting
        stored there for the same scene shape, window table, parameters and
        device is reused instead of timing, and a new result is stored."""
        import json
        import os
        key = self._cache_key()
        store = {}
        if cache and os.path.exists(cache):
            with open(cache) as f:
                store = json.load(f)
            if key in store:
                t = store[key]
                self.set_tuning(t["proj_tile"], t["gram_role_weight"])
                return dict(t, cached=True)
        Y = _cuda_f32(Y, "Y")
        if X is None:
            X = torch.empty_like(Y)
        ms = ctypes.c_float()
        _check(self.lib.hyde_windows_plan_autotune(self.plan, _ptr(Y), _ptr(X), _ptr(self.ws),
                                                   self.ws.numel(), _stream(), ctypes.byref(ms)),
               "hyde_windows_plan_autotune")
        self.graph = None
        t = dict(self.tuning(), ms=ms.value)
        if cache:
            store[key] = t
            with open(cache, "w") as f:
                json.dump(store, f, indent=1, sort_keys=True)
        return dict(t, cached=False)

    def intermediates(self) -> dict:
        """Every window's Gram matrix R [n][p][p], noise levels sigma [n][p]
        and basis V [n][p][r_max] (float64 tensors on the device) from the
        workspace, after the stream has finished."""
        from ._lib import HydeWindowsWsLayout
        lay = HydeWindowsWsLayout()
        _check(self.lib.hyde_windows_plan_layout(self.plan, ctypes.byref(lay)),
               "hyde_windows_plan_layout")
        p = self.shape[0]
        r = self.params.r_max
        n = self.n_win

        def view(off, count):
            return self.ws[off:off + 8 * count].view(torch.float64)

        return {"R": view(lay.R, n * p * p).view(n, p, p),
                "sigma": view(lay.sigma, n * p).view(n, p),
                "V": view(lay.V, n * p * r).view(n, p, r)}


class HyResWindows:
    """Sliding-window HyRes over a scene of fixed shape and window table
    (``int32[n][8]``: window y0, x0, h, w and core y0, x0, h, w). Owns the
    slot streams, fork/join events, workspace and per-window info records.
    ``__call__`` enqueues the whole scene on the current stream;
    ``capture``/``replay`` record it once into a CUDA graph and relaunch it."""

    def __init__(self, p, H, W, table, levels, r_max, n_lambda=64, n_slots=64, device="cuda",
                 lambda_mode: int = LAMBDA_SHARED, threshold_ll: bool = False):
        from ._lib import HydeWindow
        self.lib = _lib.load()
        self.shape = (p, H, W)
        self.params = params(levels, r_max, n_lambda, lambda_mode=lambda_mode,
                             threshold_ll=threshold_ll)
        self.device = torch.device(device)
        rows = [tuple(int(v) for v in r) for r in table]
        self.n_win = len(rows)
        self.win = (HydeWindow * self.n_win)(*[HydeWindow(*r) for r in rows])
        self.n_slots = min(n_slots, self.n_win)
        sz = ctypes.c_size_t()
        _check(self.lib.hyde_windows_workspace_size(p, H, W, self.win, self.n_win,
                                                    ctypes.byref(self.params), self.n_slots,
                                                    ctypes.byref(sz)),
               "hyde_windows_workspace_size")
        self.ws = _workspace(sz.value, self.device)
        self.info = torch.zeros(self.n_win * INFO_BYTES, dtype=torch.uint8, device=self.device)
        self.streams = [torch.cuda.Stream(device=self.device) for _ in range(self.n_slots)]
        self.events = [torch.cuda.Event() for _ in range(self.n_slots + 1)]
        for e in self.events:      # torch creates the CUDA event on first record
            e.record(torch.cuda.current_stream(self.device))
        torch.cuda.synchronize(self.device)
        self._streams_arr = (ctypes.c_void_p * self.n_slots)(*[s.cuda_stream for s in self.streams])
        self._events_arr = (ctypes.c_void_p * (self.n_slots + 1))(*[e.cuda_event for e in self.events])
        self.graph = None

    def __call__(self, Y: torch.Tensor, X: torch.Tensor | None = None) -> torch.Tensor:
        Y = _cuda_f32(Y, "Y")
        if tuple(Y.shape) != self.shape:
            raise ValueError(f"expected a scene of shape {self.shape}")
        if X is None:
            X = torch.empty_like(Y)
        p, H, W = self.shape
        _check(self.lib.hyde_hyres_denoise_windows(
            _ptr(Y), _ptr(X), p, H, W, self.win, self.n_win, ctypes.byref(self.params),
            _ptr(self.info), _ptr(self.ws), self.ws.numel(), self._streams_arr, self.n_slots,
            self._events_arr, _stream()), "hyde_hyres_denoise_windows")
        return X

    def capture(self, Y: torch.Tensor, X: torch.Tensor) -> None:
        """Record one scene denoise (reading Y, writing X) into a CUDA graph."""
        self(Y, X)                 # first call: function attributes, caches
        torch.cuda.synchronize(self.device)
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph, capture_error_mode="thread_local"):
            self(Y, X)

    def replay(self) -> None:
        self.graph.replay()

    def infos(self) -> list[dict]:
        raw = self.info.cpu()
        return [parse_info(raw[k * INFO_BYTES:(k + 1) * INFO_BYTES]) for k in range(self.n_win)]
