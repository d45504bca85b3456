#!/usr/bin/env python
"""Throughput benchmark of the GB300 HyRes path.

One step = one full HyRes denoise (all stages: Gram, noise regression,
eigensolver, projection, DWT, SURE selection, threshold + inverse DWT,
back-projection) of a 349 x 1905 x 144 float32 cube (the Houston-2013 shape
of the paper's experiments, Sec. 3) with 5 db2 levels, r <= 20 and K = 64
threshold candidates. The metric is Mvoxel/s (input voxels per second).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (launched by torch.distributed.run) every rank denoises its own
cube (independent replicas, no collective on the data path: weak scaling);
``value`` is all ranks' voxels over the slowest rank's time.

The reference arm (``--impl reference``) times the FP64 CPU oracle on a
bounded column slice of the same cube on the host cores.
"""

from __future__ import annotations

import argparse
import contextlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HyRes Mvoxel/s on 1 GB300 (plain vs batched/mixed, ≤1e-3 rel err); % HBM roofline"
UNIT = "Mvoxel/s"
WORKLOAD = dict(H=349, W=1905, p=144, m=12, snr_db=10.0, seed=2, levels=5, r_max=20, n_lambda=64)
L2_BYTES = 129 * 1024 * 1024
FP32_SIMT_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12   # 152 SMs x 128 FMA/clk x 2 x max clock
PAPER_A100_MVOXEL_S = 302.0   # 95.7 Mvoxel / 0.317 s (HyRes, A100, FP32, Houston 20 dB)
FP32_SM_PEAK_TFLOPS = 128 * 2 * 2.070e9 / 1e12         # one SM, for single-block kernels

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the
# dominant kernel, from one ncu capture of the 349 x 1905 x 144 cube; keyed by
# (stage, precision). profiles/ holds the capture summaries; an entry is
# removed when its kernel changes (the eigensolver has no current capture).
NCU_TRAFFIC: dict = {
    # gram_tf32 (six converter warps) 387.22 + 2.97 MB (profiles/gram_tf32_349x1905x144.md)
    ("gram", "fp32"): 390.19e6,
    ("gram", "tf32x3"): 390.19e6,
    # gram_tc 385.77 + 3.68 MB, gram_tc_reduce 8.42 MB
    ("gram", "bf16x3"): 397.87e6,
    ("gram", "bf16x3_all"): 397.87e6,
}


def _tf32_gram_flops(n: int, p: int) -> float:
    """Tensor-core flops of the split-TF32 Gram as issued: per pixel, the
    principal block (M = 128 rows, N = 32/64/128 columns) twice, and for p >
    128 the two 128 x (p' - 128) blocks three times each (p' = p rounded up
    to 16)."""
    Np = -(-p // 16) * 16
    Na = 32 if p <= 32 else 64 if p <= 64 else 128
    nb = max(Np - 128, 0)
    return 2.0 * n * 128 * (2 * Na + 6 * nb)


def _small_dense_flops(stage: str, p: int, r: int) -> float:
    """Algorithmic flops of the single-block stages: Householder
    tridiagonalisation 4p^3/3 + back-transformation of r vectors 4p^2 r
    (eig); Gauss-Jordan inverse 2p^3 (noise)."""
    if stage == "eig":
        return 4.0 * p ** 3 / 3.0 + 4.0 * p * p * r
    return 2.0 * p ** 3


def _measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return dict(hbm_gbs=float(d["hbm_gbs"]), bf16_tflops=float(d["bf16_tflops"]),
                    source="measured")
    return dict(hbm_gbs=6800.0, bf16_tflops=1900.0, source="fallback")


def _config(n_gpus: int) -> dict:
    w = WORKLOAD
    return {
        "workload": (f"HyRes denoise of a {w['H']}x{w['W']}x{w['p']} float32 synthetic cube "
                     f"(Houston-2013 shape, {w['m']} endmembers, SNR {w['snr_db']:.0f} dB), db2 "
                     f"L={w['levels']}, r<={w['r_max']}, K={w['n_lambda']}"),
        "H": w["H"], "W": w["W"], "p": w["p"], "levels": w["levels"], "r_max": w["r_max"],
        "n_lambda": w["n_lambda"], "precision": "fp32",  # replaced for --precision bf16x3
        "l2": "input 383 MB > L2, and a 256 MB buffer is written between timed steps",
        "parallelism": f"replicas x{n_gpus}",
    }


# ---------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines: list[str] = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self) -> dict:
        sm, mx, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------ CPU oracle

def _oracle_threads() -> int:
    try:
        from threadpoolctl import threadpool_info
        n = [d.get("num_threads", 0) for d in threadpool_info() if d.get("user_api") == "blas"]
        if n:
            return int(max(n))
    except Exception:
        pass
    return os.cpu_count() or 1


def oracle_sample_rate(cube, cols: int, runs: int, lambda_mode: str = "shared",
                       threshold_ll: bool = False) -> dict:
    """Time the FP64 oracle on the first ``cols`` columns of the cube."""
    import oracle as O
    w = WORKLOAD
    Ys = cube["Y"][:, :, :cols].copy()
    vox = Ys.size
    ts = []
    for _ in range(runs):
        t0 = time.perf_counter()
        O.hyres(Ys, w["levels"], w["r_max"], w["n_lambda"], lambda_mode=lambda_mode,
                threshold_ll=threshold_ll)
        ts.append(time.perf_counter() - t0)
    return dict(value=vox / 1e6 / statistics.mean(ts), times=ts, voxels=vox,
                sample=f"oracle on the {w['H']}x{cols}x{w['p']} column slice "
                       f"({vox / 1e6:.1f} Mvoxel), {runs} runs, mean time")


# --------------------------------------------------------------- bench

def _dist_setup(n_gpus: int, backend: str = "nccl"):
    """Rank layout from the launcher's environment; a process group (one
    rank per GPU, NCCL) when there is more than one rank."""
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
        return dist, world, rank, local
    return None, 1, 0, local


def _max_over_ranks(dist, values, device):
    """Element-wise maximum over the ranks of each rank's own timings: the
    job takes as long as its slowest rank."""
    vals = [float(v) for v in values]
    if dist is None:
        return vals
    import torch
    t = torch.tensor(vals, dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def _job_rate(world: int, units_per_step: float, steps: int, total_ms: float) -> float:
    """Whole-job throughput in millions of units per second: every rank
    processes ``units_per_step`` in each of ``steps`` steps (weak scaling, no
    exchange between ranks) within the slowest rank's ``total_ms``."""
    return world * units_per_step * steps / (total_ms / 1e3) / 1e6


def _stage_bytes(r_star: int) -> dict:
    w = WORKLOAD
    n = w["H"] * w["W"]
    q = 1 << w["levels"]
    N = (-(-w["H"] // q) * q) * (-(-w["W"] // q) * q)
    p, r = w["p"], w["r_max"]
    return {
        "gram": 4 * n * p,
        "project": 4 * n * p + 4 * r * N,
        "dwt": 8 * r * N,
        "sure": 4 * r * N,
        "idwt": 4 * r_star * N + 4 * r_star * n,
        "backproject": 4 * r_star * n + 4 * p * n,
    }


def _step_stats(ms) -> dict:
    """Per-step device times: mean (what value and ms_per_step use), median,
    and the olympic mean (the extremes dropped, the paper's protocol)."""
    srt = sorted(ms)
    oly = srt[1:-1] if len(srt) > 2 else srt
    return {"mean": round(statistics.mean(ms), 4), "median": round(statistics.median(ms), 4),
            "olympic": round(statistics.mean(oly), 4), "min": round(srt[0], 4),
            "max": round(srt[-1], 4), "n": len(ms)}


def _parity_full_cube(cube, X, info) -> dict:
    """The FP64 oracle on the whole timed cube, once: relative L2 error of
    the timed output, the largest per-band error, and whether the (rank,
    lambda) choice is the oracle's."""
    import numpy as np
    import oracle as O
    w = WORKLOAD
    t0 = time.perf_counter()
    o = O.hyres(cube["Y"], w["levels"], w["r_max"], w["n_lambda"])
    secs = time.perf_counter() - t0
    Xg = X.cpu().numpy().astype(np.float64)
    p = Xg.shape[0]
    d = (Xg - o["X"]).reshape(p, -1)
    band = np.linalg.norm(d, axis=1) / np.linalg.norm(o["X"].reshape(p, -1), axis=1)
    return {"rel_l2": float(O.rel_l2(Xg, o["X"])), "max_band_rel_l2": float(band.max()),
            "rank": int(info["rank"]), "lambda_index": int(info["lambda_index"]),
            "oracle_rank": int(o["rank"]), "oracle_lambda_index": int(o["k"]),
            "identical_choice": bool(int(info["rank"]) == int(o["rank"]) and
                                     int(info["lambda_index"]) == int(o["k"])),
            "oracle_sure_gap": float(o["gap"]), "oracle_seconds": round(secs, 2),
            "psnr_gain_db": float(O.psnr(cube["X"], Xg) - O.psnr(cube["X"], cube["Y"]))}


def _time_form(fn, args, flush, stream, voxels) -> dict:
    """Per-step CUDA events around fn() with the clocks sampled meanwhile."""
    clocks = ClockSampler(torch_device_index())
    with clocks:
        ms = _timed_steps(fn, args.form_steps, 3, flush, stream)
    total = float(sum(ms))
    return {"ms": round(total / len(ms), 4), "step_ms": _step_stats(ms),
            "Mvoxel/s": round(voxels * len(ms) / (total / 1e3) / 1e6, 1),
            "clocks": clocks.summary()}


def torch_device_index() -> int:
    import torch
    return torch.cuda.current_device()


def _form_precision_tf32(args, dev, cube, flush, stream) -> dict:
    """The benchmark cube with the Gram matrix on the tensor cores (split-TF32
    compensated products, FP32-accurate)."""
    return _form_precision(args, dev, cube, flush, stream, tf32=True)


def _form_precision(args, dev, cube, flush, stream, tf32: bool = False) -> dict:
    """The benchmark cube with the Gram matrix on the tensor cores (split-BF16
    compensated products, or split-TF32 with tf32), with its error against
    the FP64 oracle's Gram matrix and output."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2204_06979_gb300 import api
    w = WORKLOAD
    p, H, W = w["p"], w["H"], w["W"]
    Y = torch.from_numpy(cube["Y"]).to(dev)
    X = torch.empty_like(Y)
    h = api.HyRes(p, H, W, w["levels"], w["r_max"], w["n_lambda"], device=dev,
                  precision=api.PREC_TF32X3 if tf32 else api.PREC_BF16X3)
    out = _time_form(lambda: h(Y, X), args, flush, stream, p * H * W)
    torch.cuda.synchronize(dev)
    info = h.result_info()
    mid = h.intermediates()
    Rg = mid["R"].cpu().numpy()
    R = O.gram(cube["Y"])
    o = O.hyres(cube["Y"], w["levels"], w["r_max"], w["n_lambda"])
    Xg = X.cpu().numpy().astype(np.float64)
    d = np.sqrt(np.outer(np.diag(R), np.diag(R)))
    out.update({
        "precision": ("tf32x3 (Gram on tcgen05, split-TF32 compensated, TMEM windows of 64 "
                      "pixels added in FP32 registers)" if tf32 else
                      "bf16x3 (Gram on tcgen05, split-BF16 compensated, FP32 accumulation)"),
        "errors_vs_fp64_oracle": {
            "gram_max_rel": float(np.max(np.abs(Rg - R) / d)),
            "sigma_max_rel": float(np.max(np.abs(mid["sigma"].cpu().numpy() / o["sigma"] - 1))),
            "output_rel_l2": float(O.rel_l2(Xg, o["X"])),
            "psnr_delta_db": float(O.psnr(cube["X"], Xg) - O.psnr(cube["X"], o["X"])),
            "identical_choice": bool((info["rank"], info["lambda_index"]) ==
                                     (o["rank"], o["k"]))}})
    return out


def _form_per_level(args, dev, cube, flush, stream) -> dict:
    """The benchmark cube with one SURE threshold per kept component and
    level."""
    import torch
    from paper_2204_06979_gb300 import api
    w = WORKLOAD
    p, H, W = w["p"], w["H"], w["W"]
    Y = torch.from_numpy(cube["Y"]).to(dev)
    X = torch.empty_like(Y)
    h = api.HyRes(p, H, W, w["levels"], w["r_max"], w["n_lambda"], device=dev,
                  lambda_mode=api.LAMBDA_PER_LEVEL)
    out = _time_form(lambda: h(Y, X), args, flush, stream, p * H * W)
    info = h.result_info()
    out.update({"rank": info["rank"], "status": info["status"],
                "workload": "349x1905x144 cube, one threshold per (kept component, level)"})
    return out


def _form_diff(args, dev, cube, flush, stream) -> dict:
    """Differentiation form: 16 cubes 128 x 128 x 64, forward with learnable
    per-(component, level) threshold scales and the hand-written backward of
    an MSE-to-clean loss, one captured CUDA graph per training step."""
    import torch
    from paper_2204_06979_gb300 import api
    from synth import make_cube
    B, H, W, p, L, r = 16, 128, 128, 64, 4, 16
    cubes = [make_cube(H, W, p, m=8, seed=5 + b) for b in range(B)]
    Ys = [torch.from_numpy(cb["Y"]).to(dev) for cb in cubes]
    Xs = [torch.from_numpy(cb["X"]).to(dev) for cb in cubes]
    models = [api.HyResGrad(p, H, W, L, r, device=dev) for _ in range(B)]
    streams = [torch.cuda.Stream(dev) for _ in range(B)]
    scale = torch.ones((p, L), dtype=torch.float32, device=dev, requires_grad=True)

    def step_eager():
        scale.grad.zero_()
        Xh = api.hyres_scaled_batch(Ys, scale, models, streams)
        loss = sum(torch.mean((X_ - Xc) ** 2) for X_, Xc in zip(Xh, Xs))
        loss.backward()

    scale.grad = torch.zeros_like(scale)
    side = torch.cuda.Stream(dev)
    side.wait_stream(stream)
    with torch.cuda.stream(side):
        for _ in range(3):
            step_eager()
    stream.wait_stream(side)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        step_eager()
    out = _time_form(graph.replay, args, flush, stream, B * p * H * W)
    out.update({"workload": "16 cubes 128x128x64, db2 L=4, r<=16, forward + backward, "
                            "MSE-to-clean loss, one CUDA graph per training step",
                "grad_norm": float(scale.grad.norm())})
    return out


def _form_hyminor(args, dev, cube, flush, stream) -> dict:
    """HyMiNoR on the benchmark cube with 1 % salt-and-pepper noise added:
    HyRes, then 50 split-Bregman iterations of the l1-l1 stage; its error
    against the FP64 oracle on four bands (the bands are independent l1-l1
    problems), and against the clean cube next to HyRes alone."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2204_06979_gb300 import api
    from synth import noise as N
    w = WORKLOAD
    Yn = N.salt_and_pepper(cube["Y"], 0.01, seed=3)[0]
    Y = torch.from_numpy(Yn).to(dev)
    state = {}

    def step():
        state["X"], state["info"] = api.hyminor(Y, w["levels"], w["r_max"], w["n_lambda"])

    out = _time_form(step, args, flush, stream, Yn.size)
    torch.cuda.synchronize(dev)
    g = O.hyres(Yn, w["levels"], w["r_max"], w["n_lambda"])
    G = g["X"]
    s = float(np.max(np.abs(G)))
    bands = [0, 37, 101, 143]
    ref = s * O.tvl1_split_bregman(G[bands] / s, 1.0, 10.0, 50)
    got = state["X"].cpu().numpy()[bands].astype(np.float64)
    out.update({"workload": "349x1905x144 cube plus 1% salt-and-pepper; HyRes then 50 "
                            "split-Bregman iterations (lambda 1, mu 10)",
                "rel_l2_vs_oracle_4_bands": float(O.rel_l2(got, ref)),
                "rel_l2_to_clean_4_bands": {"hyminor": float(O.rel_l2(got, cube["X"][bands])),
                                            "hyres": float(O.rel_l2(G[bands], cube["X"][bands]))},
                "note": "time includes the workspace allocation of each call"})
    return out


def _form_forpdn(args, dev, cube, flush, stream) -> dict:
    """FORPDN on the benchmark cube (five levels, 64-point grid), with its
    error against the FP64 oracle on the whole cube and whether every
    group's smoothing choice is the oracle's."""
    import importlib
    import numpy as np
    import torch
    import oracle as O
    from paper_2204_06979_gb300 import api
    F = importlib.import_module("oracle.forpdn")
    w = WORKLOAD
    Y = torch.from_numpy(cube["Y"]).to(dev)
    state = {}

    def step():
        state["X"], state["info"] = api.forpdn(Y, w["levels"])

    out = _time_form(step, args, flush, stream, cube["Y"].size)
    torch.cuda.synchronize(dev)
    out.update({"workload": "349x1905x144 cube, db2 L=5, six groups (LL, levels 1-5), "
                            "64-point smoothing grid",
                "k": state["info"]["k"],
                "note": "time includes the workspace allocation of each call"})
    if not args.no_parity:
        ref = F.forpdn(cube["Y"], w["levels"])
        got = state["X"].cpu().numpy()
        out.update({"rel_l2_vs_oracle": float(O.rel_l2(got, ref["X"])),
                    "identical_choice": bool(list(ref["k"]) == list(state["info"]["k"])),
                    "psnr_gain_db": float(O.psnr(cube["X"], got) - O.psnr(cube["X"], cube["Y"]))})
    return out


def _form_wsrrr(args, dev, cube, flush, stream) -> dict:
    """WSRRR on the benchmark cube: HyRes, then ten cyclic-descent steps
    (thresholded coefficients, orthogonal Procrustes basis); its error
    against the FP64 oracle at the same iteration count."""
    import importlib
    import torch
    import oracle as O
    from paper_2204_06979_gb300 import api
    Wm = importlib.import_module("oracle.wsrrr")
    w = WORKLOAD
    iters = 10
    Y = torch.from_numpy(cube["Y"]).to(dev)
    state = {}

    def step():
        state["X"], state["info"] = api.wsrrr(Y, w["levels"], w["r_max"], w["n_lambda"],
                                              iters=iters)

    out = _time_form(step, args, flush, stream, cube["Y"].size)
    torch.cuda.synchronize(dev)
    out.update({"workload": "349x1905x144 cube, db2 L=5, r<=20: HyRes, then 10 WSRRR steps",
                "rank": state["info"]["rank"],
                "note": "time includes the workspace allocation of each call"})
    if not args.no_parity:
        ref = Wm.wsrrr(cube["Y"], w["levels"], w["r_max"], w["n_lambda"], iters=iters)
        got = state["X"].cpu().numpy()
        out.update({"rel_l2_vs_oracle": float(O.rel_l2(got, ref["X"])),
                    "objective_first_last": [float(ref["J"][0]), float(ref["J"][-1])],
                    "psnr_gain_db": float(O.psnr(cube["X"], got) - O.psnr(cube["X"], cube["Y"]))})
    return out


def _form_windows(args, dev, cube, flush, stream) -> dict:
    """Batched sliding-window form: a 2048 x 2048 x 200 scene in 512 uneven
    windows, every stage one launch over all windows (the plan API), replayed
    from one captured CUDA graph; the per-window pipelines on 64 streams
    (hyde_hyres_denoise_windows) beside it, and the error of sampled windows
    against the FP64 oracle."""
    import numpy as np
    import torch
    import oracle as O
    from paper_2204_06979_gb300 import api
    from synth import make_scene, make_window_table
    H = W = 2048
    p, L, r = 200, 3, 20
    T = make_window_table(H, W, depth=9, context=16, min_side=32, max_side=224, seed=4)
    sc = make_scene(H, W, p, T, m=12, seed=4)
    Yh = sc["Y"]
    Y = torch.from_numpy(Yh).to(dev)
    X = torch.zeros_like(Y)
    win = api.HyResWindowsBatched(p, H, W, T, L, r, device=dev)
    tuning = win.autotune(Y, X)   # projection tile and Gram role split, timed on this scene
    win.capture(Y, X)
    out = _time_form(win.replay, args, flush, stream, p * H * W)
    out["tuning"] = tuning
    torch.cuda.synchronize(dev)
    infos = win.infos()
    out.update({"workload": "2048x2048x200 scene, 512 windows (sides 48..256, 16-px context), "
                            "per-core SNR U[5,20] dB, db2 L=3, r<=20; 24 kernels over all "
                            "windows, one CUDA graph per scene",
                "statuses_ok": int(sum(i["status"] == 0 for i in infos)),
                "windows": len(T), "gpu_launches": win.kernel_launches,
                "l2": "the scene (3.4 GB) exceeds L2; no flush"})
    # the windows overlap (16-px context): the voxels the stages process
    win_vox = int(np.sum(T[:, 2].astype(np.int64) * T[:, 3])) * p
    out["window_voxels"] = win_vox
    out["Mvoxel/s_of_windows"] = round(win_vox / (out["ms"] / 1e3) / 1e6, 1)
    if not args.no_parity:
        areas = T[:, 2] * T[:, 3]
        picks = sorted({int(np.argmin(areas)), int(np.argmax(areas)), 16, 200, 400})
        got_all = X.cpu().numpy()
        num = den = num2 = 0.0
        same = 0
        for k in picks:
            y0, x0, h, w, cy, cx, ch, cw = (int(v) for v in T[k])
            Yk = Yh[:, y0:y0 + h, x0:x0 + w]
            o = O.hyres(Yk, L, r)
            ref = o["X"][:, cy - y0:cy - y0 + ch, cx - x0:cx - x0 + cw]
            got = got_all[:, cy:cy + ch, cx:cx + cw].astype(np.float64)
            num += float(np.sum((got - ref) ** 2))
            den += float(np.sum(ref ** 2))
            choice = (infos[k]["rank"], infos[k]["lambda_index"])
            if choice == (o["rank"], o["k"]):
                same += 1
                ref2 = ref
            else:   # a near-tie of the SURE table: the oracle at the GPU's choice
                o2 = O.hyres(Yk, L, r, rank=choice[0], lam=o["lams"][choice[1]])
                ref2 = o2["X"][:, cy - y0:cy - y0 + ch, cx - x0:cx - x0 + cw]
            num2 += float(np.sum((got - ref2) ** 2))
        out.update({"parity_windows": picks, "rel_l2_vs_oracle": float(np.sqrt(num / den)),
                    "rel_l2_vs_oracle_at_gpu_choice": float(np.sqrt(num2 / den)),
                    "identical_choice": f"{same}/{len(picks)}"})
    del win
    # the per-window pipelines (one single-cube pipeline per window, 64 streams)
    slots = api.HyResWindows(p, H, W, T, L, r, n_slots=64, device=dev)
    X2 = torch.zeros_like(Y)
    slots.capture(Y, X2)
    o2 = _time_form(slots.replay, args, flush, stream, p * H * W)
    out["per_window_pipelines"] = {"ms": o2["ms"], "Mvoxel/s": o2["Mvoxel/s"],
                                   "step_ms": o2["step_ms"]}
    return out


def run_gb300(args) -> None:
    import numpy as np
    import torch
    from paper_2204_06979_gb300 import api, _lib
    from synth import make_cube

    dist, world, rank, local = _dist_setup(args.gpus)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = WORKLOAD
    cube = make_cube(w["H"], w["W"], w["p"], m=w["m"], snr_db=w["snr_db"], seed=w["seed"])
    p, H, W = w["p"], w["H"], w["W"]
    n = H * W
    voxels = p * n
    Yd = torch.from_numpy(cube["Y"]).to(dev)
    Xd = torch.empty_like(Yd)
    prec = {"fp32": api.PREC_FP32, "tf32x3": api.PREC_TF32X3, "bf16x3": api.PREC_BF16X3,
            "bf16x3_all": api.PREC_BF16X3_ALL}[args.precision]
    lmode = {"shared": api.LAMBDA_SHARED, "per_component": api.LAMBDA_PER_COMPONENT,
             "per_level": api.LAMBDA_PER_LEVEL}[args.lambda_mode]
    h = api.HyRes(p, H, W, w["levels"], w["r_max"], w["n_lambda"], device=dev, precision=prec,
                  lambda_mode=lmode, threshold_ll=args.threshold_ll)
    lib = _lib.load()
    launches_per_step = lib.hyde_hyres_kernel_launches(p, H, W, h.params)
    if launches_per_step < 0:
        raise RuntimeError("hyde_hyres_kernel_launches rejected the workload")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize(dev)

    for _ in range(max(args.warmup, 0)):
        h(Yd, Xd)
    torch.cuda.synchronize(dev)
    info = h.result_info()

    # ---- one cube at a time (each between its own events, L2 flushed between):
    # the latency of a denoise, and the headline when --streams 1
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    slots = args.streams if (lmode == api.LAMBDA_SHARED and not args.threshold_ll) else 1
    clocks = ClockSampler(local)
    barrier()
    wall0 = time.perf_counter()
    with (clocks if slots == 1 else contextlib.nullcontext()):
        for i in range(args.steps):
            flush.fill_(float(i))
            ev[i][0].record(stream)
            h(Yd, Xd)
            ev[i][1].record(stream)
        barrier()
    wall = time.perf_counter() - wall0
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = _max_over_ranks(dist, [sum(step_ms)], dev)[0]
    ms_per_step = total_ms / args.steps
    value = _job_rate(world, voxels, args.steps, total_ms)
    step_stats = _step_stats(step_ms)
    latency = {"ms": round(ms_per_step, 4), "step_ms": step_stats,
               "value": round(value, 1)}
    X_timed = Xd.clone() if rank == 0 else None

    # ---- the headline: K cubes in flight over `slots` workspaces and streams
    # (hyde_hyres_denoise_many), distinct input copies (each 383 MB > L2, so
    # no flush is needed between them), exactly K cubes between a barrier +
    # synchronize on both sides
    pipeline = None
    if slots > 1:
        many = api.HyResMany(p, H, W, w["levels"], w["r_max"], w["n_lambda"], slots=slots,
                             device=dev, precision=prec)
        Ys = [Yd] + [Yd.clone() for _ in range(slots - 1)]
        Xs = [torch.empty_like(Yd) for _ in range(slots)]
        pick = lambda K: ([Ys[k % slots] for k in range(K)], [Xs[k % slots] for k in range(K)])
        if args.warmup > 0:
            many(*pick(args.warmup))
        torch.cuda.synchronize(dev)
        yk, xk = pick(args.steps)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier()
        wall0 = time.perf_counter()
        with clocks:
            e0.record(stream)
            many(yk, xk)
            e1.record(stream)
            barrier()
        wall = time.perf_counter() - wall0
        total_ms = _max_over_ranks(dist, [e0.elapsed_time(e1)], dev)[0]
        ms_per_step = total_ms / args.steps
        value = _job_rate(world, voxels, args.steps, total_ms)
        X_timed = Xs[(args.steps - 1) % slots].clone() if rank == 0 else None
        last = many.result_info(args.steps - 1)
        pipeline = {"slots": slots, "ms_per_cube": round(ms_per_step, 4),
                    "last_cube_status": last["status"], "last_cube_rank": last["rank"],
                    "identical_to_serial": bool(torch.equal(Xs[(args.steps - 1) % slots], Xd))}

    # ---- per-stage timing through the timed entry point (same launches)
    nst = _lib.N_STAGES
    stage_ev = [[torch.cuda.Event(enable_timing=True) for _ in range(nst + 1)]
                for _ in range(args.steps)]
    for row in stage_ev:          # torch creates the CUDA event on first record
        for e in row:
            e.record(stream)
    torch.cuda.synchronize(dev)
    import ctypes
    stage_ms = {name: [] for name in _lib.STAGE_NAMES}
    for i in range(args.steps):
        flush.fill_(float(i))
        arr = (ctypes.c_void_p * (nst + 1))(*[e.cuda_event for e in stage_ev[i]])
        code = lib.hyde_hyres_denoise_timed(
            Yd.data_ptr(), Xd.data_ptr(), p, H, W, ctypes.byref(h.params), h.info.data_ptr(),
            h.ws.data_ptr(), h.ws.numel(), stream.cuda_stream, arr)
        if code != 0:
            raise RuntimeError(f"hyde_hyres_denoise_timed failed: {code}")
    torch.cuda.synchronize(dev)
    for i in range(args.steps):
        for s, name in enumerate(_lib.STAGE_NAMES):
            stage_ms[name].append(stage_ev[i][s].elapsed_time(stage_ev[i][s + 1]))
    stage_avg = {k: statistics.mean(v) for k, v in stage_ms.items()}
    info = h.result_info()
    r_star = int(info["rank"])
    peaks = _measured_peaks()
    sbytes = _stage_bytes(r_star)
    dominant = max(stage_avg, key=stage_avg.get)
    if dominant == "gram" and args.precision in ("tf32x3", "fp32") and p % 4 == 0 and p <= 160:
        # tf32 MMA work per pixel: the principal 128-band block twice (H H^T and
        # H (2L)^T), the other band blocks three times; tensor peak for tf32 is
        # half the measured bf16 rate
        flops = _tf32_gram_flops(n, p)
        tc_peak = peaks["bf16_tflops"] / 2
        achieved = flops / (stage_avg["gram"] / 1e3) / 1e12
        bts = sbytes["gram"]
        roofline = {"kernel": "gram_tf32 (tcgen05 split-TF32, TMA) + reduce", "bound": "hbm",
                    "achieved": bts / (stage_avg["gram"] / 1e3) / 1e9, "peak": peaks["hbm_gbs"],
                    "unit": "GB/s", "frac": bts / (stage_avg["gram"] / 1e3) / 1e9 / peaks["hbm_gbs"],
                    "peak_source": peaks["source"],
                    "algorithmic": f"{bts} bytes per launch (4 B per voxel read)",
                    "tensor": {"achieved_tflops": achieved, "peak_tflops": tc_peak,
                               "frac": achieved / tc_peak,
                               "peak_source": "measured bf16 burst / 2 (tf32 rate)",
                               "flops": flops}}
    elif dominant == "gram" and args.precision != "fp32":
        flops = 3 * 2 * n * p * p   # three bf16 products per entry (hi hi, hi lo, lo hi)
        tc_peak = peaks["bf16_tflops"]
        achieved = flops / (stage_avg["gram"] / 1e3) / 1e12
        roofline = {"kernel": "gram_tc (tcgen05 split-BF16) + reduce", "bound": "tensor",
                    "achieved": achieved, "peak": tc_peak, "unit": "TFLOP/s",
                    "frac": achieved / tc_peak,
                    "peak_source": peaks["source"] + " bf16 dense (burst)",
                    "algorithmic": f"{flops:.4g} flop per launch (3 products of 2np^2)"}
    elif dominant == "gram":
        flops = n * p * (p + 1)   # the symmetric product computed: n p (p+1)/2 FMAs
        achieved = flops / (stage_avg["gram"] / 1e3) / 1e12
        roofline = {"kernel": "gram (gram_partial + gram_reduce)", "bound": "alu",
                    "achieved": achieved, "peak": FP32_SIMT_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_SIMT_PEAK_TFLOPS,
                    "peak_source": "derived: 152 SMs x 128 FP32 FMA/clk x 2 x 2070 MHz",
                    "algorithmic": f"{flops:.4g} flop per launch"}
    elif dominant in sbytes:
        bts = sbytes[dominant]
        achieved = bts / (stage_avg[dominant] / 1e3) / 1e9
        roofline = {"kernel": dominant, "bound": "hbm", "achieved": achieved,
                    "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": achieved / peaks["hbm_gbs"],
                    "peak_source": peaks["source"],
                    "algorithmic": f"{bts} bytes per launch"}
    else:
        # eig / noise: one thread block by construction (a p x p problem),
        # bound by the dependent chain of its p steps, so the ceiling that
        # applies is one SM's FP32 rate; the whole-GPU fraction is also given
        flops = _small_dense_flops(dominant, p, w["r_max"])
        achieved = flops / (stage_avg[dominant] / 1e3) / 1e12
        roofline = {"kernel": dominant, "bound": "alu", "achieved": achieved,
                    "peak": FP32_SM_PEAK_TFLOPS, "unit": "TFLOP/s",
                    "frac": achieved / FP32_SM_PEAK_TFLOPS,
                    "frac_of_gpu": achieved / FP32_SIMT_PEAK_TFLOPS,
                    "peak_source": "derived: 1 SM x 128 FP32 FMA/clk x 2 x 2070 MHz "
                                   "(single-block kernel)",
                    "algorithmic": f"{flops:.4g} flop per launch"}
    roofline["traffic"] = NCU_TRAFFIC.get((dominant, args.precision))
    hbm_stages = {}
    for k, bts in sbytes.items():
        gbs = bts / (stage_avg[k] / 1e3) / 1e9
        hbm_stages[k] = {"ms": round(stage_avg[k], 4), "GB/s": round(gbs, 1),
                         "frac_hbm": round(gbs / peaks["hbm_gbs"], 3)}

    # ---- end to end through the public call with host buffers: a stream of
    # args.steps cubes in page-locked host memory, each copied in, denoised and
    # copied out (with its info record) by hyde_hyres_denoise_host, which
    # overlaps the copies of the neighbouring cubes with each denoise; the
    # same cubes one after another on one stream are reported beside it
    Yh = torch.from_numpy(cube["Y"]).pin_memory()
    Xh = [torch.empty_like(Yh).pin_memory() for _ in range(2)]
    info_h = torch.empty(args.steps * h.info.numel(), dtype=torch.uint8).pin_memory()
    Ys = [Yh] * args.steps
    Xs = [Xh[i & 1] for i in range(args.steps)]
    h.denoise_host(Ys[:2] if args.steps >= 2 else Ys, Xs[:2] if args.steps >= 2 else Xs)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    h.denoise_host(Ys, Xs, info_h)
    e1.record(stream)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    # the same, serialised on one stream
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for i in range(args.steps):
        Yd.copy_(Yh, non_blocking=True)
        h(Yd, Xd)
        Xh[0].copy_(Xd, non_blocking=True)
        info_h[:h.info.numel()].copy_(h.info, non_blocking=True)
    s1.record(stream)
    barrier()
    serial_ms = s0.elapsed_time(s1)
    e2e_ms, serial_ms = _max_over_ranks(dist, [e2e_ms, serial_ms], dev)
    e2e_value = _job_rate(world, voxels, args.steps, e2e_ms)
    e2e_serial = _job_rate(world, voxels, args.steps, serial_ms)

    # ---- parity of the timed output against the FP64 oracle on the whole cube
    parity = None
    if rank == 0 and world == 1 and not args.no_parity:
        parity = _parity_full_cube(cube, X_timed, info)

    # ---- the other forms, each on its own workload (rank 0 of a 1-GPU run)
    forms = None
    if rank == 0 and world == 1 and not args.no_forms:
        forms = {}
        for name, fn in (("precision_tf32x3", _form_precision_tf32),
                         ("precision_bf16x3", _form_precision), ("per_level", _form_per_level),
                         ("diff", _form_diff), ("hyminor", _form_hyminor),
                         ("forpdn", _form_forpdn), ("wsrrr", _form_wsrrr),
                         ("windows", _form_windows)):
            try:
                forms[name] = fn(args, dev, cube, flush, stream)
            except Exception as exc:   # a failing form is reported, not hidden
                forms[name] = {"error": f"{type(exc).__name__}: {exc}"}

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        s = oracle_sample_rate(cube, cols=args.cpu_cols, runs=args.cpu_runs,
                               lambda_mode=args.lambda_mode, threshold_ll=args.threshold_ll)
        cpu = {"value": round(s["value"], 3), "unit": UNIT, "cores": _oracle_threads(),
               "kind": "oracle", "sample": s["sample"]}

    if rank == 0:
        cfg = _config(world)
        if pipeline is not None:
            cfg["streams"] = slots
            cfg["workload"] += (f", {slots} cubes in flight (hyde_hyres_denoise_many: one "
                                f"workspace and stream each)")
            cfg["l2"] = (f"each cube's input (383 MB, {slots} distinct copies) exceeds L2; no "
                         f"flush between pipelined cubes (the serial latency run flushes 256 MB "
                         f"between steps)")
        if args.precision == "tf32x3":
            cfg["precision"] = "tf32x3 (Gram on tcgen05, split-TF32 compensated, FP32-accurate)"
            cfg["workload"] += ", Gram on the tensor cores (split-TF32)"
        elif args.precision == "bf16x3":
            cfg["precision"] = "bf16x3 (Gram on tcgen05, split-BF16 compensated)"
            cfg["workload"] += ", precision form"
        elif args.precision == "bf16x3_all":
            cfg["precision"] = ("bf16x3_all (Gram, projection and back-projection on tcgen05, "
                                "split-BF16 compensated)")
            cfg["workload"] += ", precision form (all contractions on the tensor cores)"
        if args.lambda_mode == "per_component":
            cfg["lambda_mode"] = "per_component (one SURE threshold per kept component)"
            cfg["workload"] += ", per-component thresholds"
        elif args.lambda_mode == "per_level":
            cfg["lambda_mode"] = "per_level (one SURE threshold per kept component and level)"
            cfg["workload"] += ", per-level thresholds"
        if args.threshold_ll:
            cfg["threshold_ll"] = True
            cfg["workload"] += ", final LL band thresholded too"
        line = {
            "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_per_step, 4),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp32": "f32", "tf32x3": "tf32x3+f32"}.get(args.precision, "bf16x3+f32"),
            "data": "synthetic", "config": cfg,
            "roofline": roofline,
            "stages": hbm_stages | {k: {"ms": round(v, 4)} for k, v in stage_avg.items()
                                    if k not in hbm_stages},
            "e2e": {"value": round(e2e_value, 1), "unit": UNIT,
                    "h2d_bytes_per_step": int(Yh.numel() * 4),
                    "d2h_bytes_per_step": int(Yh.numel() * 4 + h.info.numel()),
                    "mode": "hyde_hyres_denoise_host: cube s+1 copied in and cube s-1 out "
                            "while cube s is denoised",
                    "serial_value": round(e2e_serial, 1)},
            "gpu_launches": int(launches_per_step * args.steps),
            "step_ms": step_stats if pipeline is None else None,
            "latency": latency,
            "pipeline": pipeline,
            "parity": parity,
            "forms": forms,
            "clocks": clocks.summary(),
            "cpu_baseline": cpu,
            "selection": {"rank": r_star, "lambda_index": info["lambda_index"],
                          "status": info["status"]},
            "wall_s_timed": round(wall, 3),
            "context": {"paper_a100_fp32_mvoxel_s": PAPER_A100_MVOXEL_S,
                        "note": "paper: HyRes on the real Houston cube at 20 dB on an A100 "
                                "(0.317 s); context only"},
        }
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    _ = np


def _timed_steps(fn, steps, warmup, flush, stream):
    """Per-step CUDA events around fn(), an L2-flushing write between steps."""
    import torch
    for _ in range(max(warmup, 0)):
        fn()
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        ev[i][0].record(stream)
        fn()
        ev[i][1].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev]


def run_form(args) -> None:
    """Secondary workloads: the batched sliding-window form and the
    differentiation form (one JSON line each; not the headline metric)."""
    import numpy as np
    import torch
    from paper_2204_06979_gb300 import api
    from synth import make_cube, make_scene, make_window_table

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    peaks = _measured_peaks()
    clocks = ClockSampler(0)
    if args.form == "windows":
        H = W = args.win_scene
        p, L, r = 200, 3, 20
        # the 2048 x 2048 scene has 2^9 windows; a quarter of the area, a quarter of them
        depth = {2048: 9, 1024: 7, 512: 5}[H]
        T = make_window_table(H, W, depth=depth, context=16, min_side=32, max_side=224, seed=4)
        sc = make_scene(H, W, p, T, m=12, seed=4)
        Y = torch.from_numpy(sc["Y"]).to(dev)
        X = torch.zeros_like(Y)
        if args.slots > 0:   # the per-window pipelines on that many streams
            win = api.HyResWindows(p, H, W, T, L, r, n_slots=args.slots, device=dev)
        else:                # every stage one launch over all windows, tuned on the scene
            win = api.HyResWindowsBatched(p, H, W, T, L, r, device=dev)
            win.autotune(Y, X)
        win.capture(Y, X)
        with clocks:
            ms = _timed_steps(win.replay, args.steps, args.warmup, flush, stream)
        voxels = p * H * W
        infos = win.infos()
        extra = {"windows": len(T), "slots": args.slots if args.slots > 0 else "batched",
                 "window_sides": [int(T[:, 2:4].min()), int(T[:, 2:4].max())],
                 "statuses_ok": int(sum(i["status"] == 0 for i in infos)),
                 "ranks": [int(min(i["rank"] for i in infos)), int(max(i["rank"] for i in infos))]}
        # bytes the windows touch at least: read their cubes twice (Gram,
        # projection) and write the scene once
        win_vox = int(np.sum(T[:, 2].astype(np.int64) * T[:, 3]) * p)
        alg_bytes = 4 * (2 * win_vox + voxels)
        workload = (f"sliding-window HyRes of a {H}x{W}x200 float32 synthetic scene, {len(T)} "
                    "uneven windows (sides 48..256, 16-px context), per-core SNR U[5,20] dB, "
                    "db2 L=3, r<=20, K=64, one captured CUDA graph per scene")
    else:
        B, H, W, p, L, r = 16, 128, 128, 64, 4, 16
        cubes = [make_cube(H, W, p, m=8, seed=5 + b) for b in range(B)]
        Ys = [torch.from_numpy(cb["Y"]).to(dev) for cb in cubes]
        Xs = [torch.from_numpy(cb["X"]).to(dev) for cb in cubes]
        models = [api.HyResGrad(p, H, W, L, r, device=dev) for _ in range(B)]
        streams = [torch.cuda.Stream(dev) for _ in range(B)]
        scale = torch.ones((p, L), dtype=torch.float32, device=dev, requires_grad=True)

        def step_eager():
            # every cube's forward and backward on its own stream
            scale.grad.zero_()
            Xh = api.hyres_scaled_batch(Ys, scale, models, streams, sm_cap=args.sm_cap)
            loss = sum(torch.mean((X_ - Xc) ** 2) for X_, Xc in zip(Xh, Xs))
            loss.backward()

        # the whole training step (forward, loss, backward, gradient zeroing)
        # captured once into a CUDA graph: 16 small cubes are bound by the
        # host's launch rate otherwise
        scale.grad = torch.zeros_like(scale)
        side = torch.cuda.Stream(dev)
        side.wait_stream(stream)
        with torch.cuda.stream(side):
            for _ in range(3):
                step_eager()
        stream.wait_stream(side)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph):
            step_eager()
        with clocks:
            ms = _timed_steps(graph.replay, args.steps, args.warmup, flush, stream)
        voxels = B * p * H * W
        extra = {"batch": B, "loss": "MSE to clean", "grad_norm": float(scale.grad.norm()),
                 "launch": "one CUDA graph per training step, one stream per cube"}
        # forward (3 cube passes) + backward (2 cube reads) per cube
        alg_bytes = 4 * 5 * voxels
        workload = ("differentiation form: forward + hand-written backward of HyRes with "
                    "learnable 64x4 threshold scales on a batch of 16 synthetic 128x128x64 "
                    "cubes, MSE-to-clean loss, db2 L=4, r<=16")
    total_ms = float(sum(ms))
    value = voxels * len(ms) / (total_ms / 1e3) / 1e6
    achieved = alg_bytes / (total_ms / len(ms) / 1e3) / 1e9
    line = {
        "metric": METRIC, "value": round(value, 1), "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(total_ms / len(ms), 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic", "config": {"workload": workload, "form": args.form,
                                        "l2": "inputs larger than L2 and a 256 MB write between steps"},
        "roofline": {"kernel": "whole step (effective)", "bound": "hbm", "achieved": achieved,
                     "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": achieved / peaks["hbm_gbs"], "traffic": None,
                     "algorithmic": f"{alg_bytes} bytes per step"},
        "clocks": clocks.summary(), "form_details": extra,
    }
    print(json.dumps(line), flush=True)


def run_reference(args) -> None:
    from synth import make_cube
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = WORKLOAD
    cube = make_cube(w["H"], w["W"], w["p"], m=w["m"], snr_db=w["snr_db"], seed=w["seed"])
    import oracle as O
    Ys = cube["Y"][:, :, :args.cpu_cols].copy()
    for _ in range(max(args.warmup, 0)):
        O.hyres(Ys, w["levels"], w["r_max"], w["n_lambda"])
    ts = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        O.hyres(Ys, w["levels"], w["r_max"], w["n_lambda"])
        ts.append(time.perf_counter() - t0)
    vox = Ys.size
    value = vox * len(ts) / sum(ts) / 1e6
    sample = (f"FP64 numpy oracle on the {w['H']}x{args.cpu_cols}x{w['p']} column slice "
              f"({vox / 1e6:.1f} Mvoxel) of the cube, one slice per step")
    line = {
        "impl": "reference", "metric": METRIC, "value": round(value, 3), "unit": UNIT,
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(1e3 * sum(ts) / len(ts), 2), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": _config(world),
        "cpu_baseline": {"value": round(value, 3), "unit": UNIT, "cores": _oracle_threads(),
                         "kind": "oracle", "sample": sample},
        "e2e": {"value": round(value, 3), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def main() -> None:
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--streams", type=int, default=4,
                    help="cubes in flight for the headline (hyde_hyres_denoise_many); 1 = one "
                         "cube at a time")
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=("gb300", "reference"), default="gb300")
    ap.add_argument("--cpu-cols", type=int, default=384,
                    help="columns of the cube in the CPU oracle sample")
    ap.add_argument("--cpu-runs", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-parity", action="store_true",
                    help="skip the FP64 oracle run on the whole timed cube")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the precision, per-level, differentiation and window forms")
    ap.add_argument("--form-steps", type=int, default=5,
                    help="timed steps of each secondary form in the plain run")
    ap.add_argument("--form", choices=("plain", "windows", "diff"), default="plain",
                    help="plain: the headline workload; windows / diff: secondary forms")
    ap.add_argument("--win-scene", type=int, default=2048, choices=(2048, 1024, 512),
                    help="--form windows: scene side (2048: the benchmark scene; smaller "
                         "sides for profiler captures)")
    ap.add_argument("--slots", type=int, default=0,
                    help="--form windows: 0 runs every stage once over all windows (the "
                         "batched plan); n > 0 the per-window pipelines on n streams")
    ap.add_argument("--sm-cap", type=int, default=None,
                    help="--form diff: SMs each cube's grids are sized for (0: all; "
                         "default: the batch API's choice)")
    ap.add_argument("--precision", choices=("fp32", "tf32x3", "bf16x3", "bf16x3_all"),
                    default="fp32",
                    help="fp32: plain form (headline); tf32x3: Gram on the tensor cores, "
                         "split-TF32 (FP32-accurate); bf16x3: Gram on the tensor cores, "
                         "split-BF16; bf16x3_all: the projections there too")
    ap.add_argument("--lambda-mode", choices=("shared", "per_component", "per_level"),
                    default="shared",
                    help="shared: one SURE threshold for every kept component (headline); "
                         "per_component: each kept component at its own threshold; "
                         "per_level: each kept component and level at its own threshold")
    ap.add_argument("--threshold-ll", action="store_true",
                    help="soft-threshold (and count in SURE) the final LL band too")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "gb300":
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.form != "plain":
        run_form(args)
    else:
        run_gb300(args)


if __name__ == "__main__":
    main()
