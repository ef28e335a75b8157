"""Benchmark: SARA-SDMM on one GB300 (1024^2 sky, 4,194,304 uv points).

One step = one SDMM iteration (Algorithm 1): the CG global update with 10
conjugate-gradient steps (11 applications of Re Phi^H Phi + 2I), the l1 block
on Psi^H x (analysis with the fused prox), the positivity block, the l2-ball
block (Phi, projection, Phi^H) -- every kernel of the hot path.

Prints one JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
on the host cores instead: real oracle SDMM iterations of the same workload,
as many as fit a bounded time (``steps`` reports how many were timed).
Under torchrun every rank runs its own independent solve (replicas, weak
scaling); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "SDMM iters/s & Phi+Phi^H vis/s at 1024^2,M=4M vs plain GPU; solves/s, p99 latency"
UNIT = "iters/s"
WORKLOAD = "large_1024"
# DRAM bytes (read + write) per launch from the committed ncu capture of each
# kernel at this workload (profiles/); kernels changed since have no entry.
MEASURED_TRAFFIC = {"col_conv": 16.84224e6 + 0.0}


# ----------------------------------------------------------------- helpers
def dist_info():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(ms: float, pg, dev) -> float:
    """The slowest rank's time (all-reduce MAX over the process group; the
    local time when there is no group)."""
    if pg is None:
        return ms
    import torch

    t = torch.tensor([ms], device=dev, dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, ws: int, ms: float) -> float:
    """Units all ranks processed per second over the slowest rank's time."""
    return units_per_rank * ws / (ms / 1e3)


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(self.gpu)], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.t.join(timeout=2)

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm), "window": "the same SDMM iterations for ~0.6 s, then the timed region"}


def workload_string(name: str, w) -> str:
    """The workload description both arms print in config.workload."""
    return (f"{name}: {w.n}x{w.n} sky, M={w.M} uv points, {2 * w.n}^2 grid, J=8, SARA {w.levels} levels, "
            f"{w.cg_iters} CG steps per iteration")


def algorithmic_bytes(kind: str, n: int, M: int, rsize: int = 4, levels: int = 4, cg: int = 10) -> float:
    """Bytes each kernel kind must move per launch (FP32: 4-byte reals, 8-byte
    complex).  N = n^2 pixels; the oversampled grid holds 4N complex cells.
    The SARA sets count one launch set (all levels) in their SDMM form:
    analysis with the l1 prox (x in; z_1, w in, z_1 and 2r - v out for the
    9N coefficients; LL scratch bands out and in level by level), synthesis
    with the positivity block (2r - v in, scratch bands, x_hat and z_2 in,
    z_2 and x_1 + x_2 out)."""
    N = n * n
    c = 2 * rsize
    band = sum(8 * (N >> (2 * lev)) for lev in range(1, levels))  # 8 filters' LL bands of levels 1..L-1
    table = {
        "sara_analysis": N * rsize + 9 * N * 4 * rsize + 2 * band * rsize,
        "sara_synthesis": 9 * N * rsize + 2 * band * rsize + 4 * N * rsize,
        "gram": 4 * N * c * 2 + 8 * M,          # read grid, write grid accumulator, read positions
        "degrid": 4 * N * c + 8 * M + 3 * c * M,  # grid + positions + (z read, y read, z write)
        "grid": 4 * N * c + 8 * M + 3 * c * M,    # grid write + positions + (z, y read, z write)
        # Phi / Phi^H in real form: half-spectrum rows n x n complex
        "row_fwd": N * rsize + N * c,             # image in, half-spectrum rows out
        "col_fwd": N * c + 4 * N * c,             # half-spectrum rows in, full grid out
        "col_inv": 4 * N * c + N * c,             # accumulator in, half-spectrum rows out
        "row_inv": N * c + 2 * N * rsize,         # half-spectrum rows in, image in/out (epilogue)
        # convolution form (real image, half spectra n x n complex), averaged
        # over the cg + 1 launches per SDMM iteration: the CG's first forward
        # pass forms r = p = b - A x_hat (b, A x_hat in; r, p out), the other
        # cg - 1 apply the CG update (x, r, p, Ap in; x, r, p out), and the
        # pass of A x_hat for the next CG start reads x_hat; the cg inverse
        # passes of the CG form Ap (p, r in; Ap out), the one of A x_hat
        # reads x_hat and writes A x_hat
        "row_fwd_h": ((4 * N * rsize + N * c) + (cg - 1) * (7 * N * rsize + N * c) + (N * rsize + N * c)) / (cg + 1),
        "col_conv": N * c + 2 * N * rsize + N * c,  # half-spectrum rows in, PSF half spectrum, rows out
        "row_inv_h": (cg * (N * c + 3 * N * rsize) + (N * c + 2 * N * rsize)) / (cg + 1),
    }
    return float(table.get(kind, 0))


# ----------------------------------------------------------------- our arm
def run_ours(args, ws, rank, local):
    import numpy as np
    import torch

    from paper_1406_0359_gb300 import build as _build
    from paper_1406_0359_gb300 import synth
    from paper_1406_0359_gb300.binding import KERNEL_KINDS, Operator

    _build.build()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    w = synth.WORKLOADS[args.workload]
    n, M, L = w.n, w.M, w.levels
    seed = w.seed + 1000 * rank
    uv_h = synth.uv_coverage(M, n, seed)
    x_h = synth.sky(n, seed, w.n_blobs, w.n_points)
    a_h, b_h = synth.noise_draws(M, seed)

    pg = None
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
        pg = dist

    def barrier():
        if pg:
            pg.barrier()
        torch.cuda.synchronize()

    uv = torch.as_tensor(uv_h, device=dev)
    from paper_1406_0359_gb300.binding import purify_autotune

    if args.tile and args.chunk:  # fixed work decomposition (reproducible profiles)
        tile, chunk, tune_ms = args.tile, args.chunk, None
    else:
        tile, chunk, tune_ms = purify_autotune(uv, n, L)
    op = Operator(uv, n, L, "fp32", tile=tile, chunk=chunk)
    info = op.info()
    xt = torch.as_tensor(x_h, dtype=torch.float32, device=dev)
    y0 = op.phi(xt)
    sigma = float(torch.linalg.vector_norm(y0.to(torch.complex128))) / math.sqrt(M) * 10 ** (-w.isnr_db / 20)
    noise = torch.complex(torch.as_tensor(a_h), torch.as_tensor(b_h)).to(dev, torch.complex64)
    y = (y0 + (sigma / math.sqrt(2)) * noise).contiguous()
    eps = sigma * math.sqrt(M + 2 * math.sqrt(M))

    # nu, gamma by the library's own rules (power iteration, backprojection)
    r0 = op.solve(y, eps, t_max=1, cg_iters=1)
    nu, gamma = r0.stats["nu"], r0.stats["gamma"]
    kw = dict(t_max=args.warmup, cg_iters=w.cg_iters, gamma=gamma, nu=nu)
    op.solve(y, eps, **kw)  # warm-up: W SDMM iterations

    K = args.steps
    kw["t_max"] = K
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        # nvidia-smi samples every 200 ms, longer than a short timed region:
        # keep the GPU on the same iterations for ~0.6 s first, so that the
        # samples describe the clocks under this load up to the timed region
        t_load = time.perf_counter() + 0.6
        while time.perf_counter() < t_load:
            op.solve(y, eps, **dict(kw, t_max=max(K, 20)))
            torch.cuda.synchronize()
        barrier()
        torch.cuda.nvtx.range_push("sdmm_timed")  # scopes ncu captures to the timed iterations
        e0.record()
        res = op.solve(y, eps, **kw)
        e1.record()
        torch.cuda.nvtx.range_pop()
        barrier()
    ms = max_over_ranks(e0.elapsed_time(e1), pg, dev)
    value = whole_job_rate(K, ws, ms)

    # profiled pass of the same K steps: per-kernel device time (CUDA events on the solver's stream)
    op.profile(True)
    op.solve(y, eps, **kw)
    kt = op.kernel_times()
    op.profile(False)
    busy = {k: v for k, v in kt.items() if v[1] > 0 and k != "memset"}
    total_busy = sum(v[0] for v in busy.values())
    dom = max(busy, key=lambda k: busy[k][0])
    dom_ms, dom_n = busy[dom]
    hbm, peak_kind = peaks()
    bytes_launch = algorithmic_bytes(dom, n, M, levels=L, cg=w.cg_iters)
    achieved = bytes_launch / (dom_ms / dom_n / 1e3) / 1e9
    kernels_per_call = {"sara_analysis": 1 + L, "sara_synthesis": L}
    launches = sum(v[1] * kernels_per_call.get(k, 1) for k, v in kt.items() if k != "memset")
    per_kernel = {}
    for k, v in busy.items():
        e = {"ms_per_launch": round(v[0] / v[1], 4), "launches": v[1], "share": round(v[0] / total_busy, 4)}
        b = algorithmic_bytes(k, n, M, levels=L, cg=w.cg_iters)
        if b > 0:  # achieved algorithmic GB/s and its fraction of the measured HBM copy peak
            gbs = b / (v[0] / v[1] / 1e3) / 1e9
            e.update({"bytes_per_launch": b, "gbs": round(gbs, 1), "frac_of_hbm_peak": round(gbs / hbm, 4)})
        per_kernel[k] = e

    # Phi + Phi^H throughput (visibilities per second)
    reps = max(3, K // 2)
    for _ in range(2):
        op.phi_adj(op.phi(xt))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        op.phi_adj(op.phi(xt))
    e1.record()
    torch.cuda.synchronize()
    pair_ms = e0.elapsed_time(e1) / reps
    vis_per_s = M / (pair_ms / 1e3)
    # bytes of one Phi + Phi^H pair: the staged count (every pass's reads and
    # writes, FP32: Phi 196N + 16M, Phi^H 204N + 16M) and the compulsory one
    # (image in and out, uv positions and visibilities once: 2 (4N + 16M))
    N = n * n
    pair_bytes = {"staged": float(400 * N + 32 * M), "compulsory": float(8 * N + 32 * M)}
    pair_gbs = {k: round(v / (pair_ms / 1e3) / 1e9, 1) for k, v in pair_bytes.items()}

    # end to end through the public API from pinned host buffers
    from paper_1406_0359_gb300.binding import Operator as Op2

    uv_pin = torch.as_tensor(uv_h).pin_memory()
    y_pin = y.cpu().pin_memory()
    x_pin = torch.empty(n, n, dtype=torch.float32).pin_memory()
    side = torch.cuda.Stream(dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    uv_d = uv_pin.to(dev, non_blocking=True)
    with torch.cuda.stream(side):  # y travels while the operator is built from uv
        y_d = y_pin.to(dev, non_blocking=True)
    op2 = Op2(uv_d, n, L, "fp32")
    torch.cuda.current_stream().wait_stream(side)
    r2 = op2.solve(y_d, eps, **kw)
    x_pin.copy_(r2.x, non_blocking=True)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    op2.close()
    e2e = {"value": round(K / e2e_s, 3), "unit": UNIT,
           "h2d_bytes_per_step": int((uv_pin.numel() * 8 + y_pin.numel() * 8) / K),
           "d2h_bytes_per_step": int(x_pin.numel() * 4 / K),
           "includes": "H2D of uv, then operator creation (uv binning) beside the H2D of y, K SDMM iterations, "
                       "D2H of x; per solve / K"}

    # plain FP64 GPU solver (no graph), same problem; and the precision study:
    # FP32 (compensated gridding, FP64 reductions) against FP64 on the GPU,
    # per operator and for the image after the same iterations
    plain = None
    precision = None
    if not args.no_plain:
        op64 = Operator(uv, n, L, "fp64")
        y64 = y.to(torch.complex128)
        kp = max(2, K // 4)
        op64.solve(y64, eps, t_max=1, cg_iters=w.cg_iters, gamma=gamma, nu=nu, use_graph=False)
        torch.cuda.synchronize()
        e0.record()
        r64 = op64.solve(y64, eps, t_max=kp, cg_iters=w.cg_iters, gamma=gamma, nu=nu, use_graph=False)
        e1.record()
        torch.cuda.synchronize()
        plain = kp / (e0.elapsed_time(e1) / 1e3)

        def rel(a, b):
            a, b = a.to(torch.complex128 if b.is_complex() else torch.float64), b
            return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))

        x64 = xt.to(torch.float64)
        r32 = op.solve(y, eps, t_max=kp, cg_iters=w.cg_iters, gamma=gamma, nu=nu)
        precision = {"phi": rel(op.phi(xt), op64.phi(x64)), "phi_adj": rel(op.phi_adj(y), op64.phi_adj(y64)),
                     "psi_h": rel(op.sara_fwd(xt), op64.sara_fwd(x64)),
                     "image_after_%d_iters" % kp: rel(r32.x, r64.x),
                     "reference": "same operators and solver in FP64 on the GPU"}
        op64.close()

    batch = None
    if rank == 0 and not args.no_batch_summary:
        batch = batch_study(16, 20, seed=40, plain_arm=False)
        batch["note"] = "reduced form of the 64-instance batch (bench.py --batch); solves/s of 16 instances x 20 iterations"

    serving = None
    if rank == 0 and not args.no_batch_summary:
        serving = serving_summary()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        y1 = op.phi(xt)
        gpu_out = {"phi": y1.cpu().numpy().astype(np.complex128),
                   "phi_adj_phi": op.phi_adj(y1).cpu().numpy().astype(np.float64),
                   "psi_h": op.sara_fwd(xt).cpu().numpy().astype(np.float64)}
        cpu = cpu_baseline(args.workload, gpu=gpu_out)

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": ws, "steps": K,
        "warmup": args.warmup, "ms_per_step": round(ms / K, 4), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32 (compensated reductions, FP64 finals)", "data": "synthetic",
        "config": {"workload": workload_string(args.workload, w),
                   "global_batch": ws, "parallelism": f"replicas x{ws}",
                   "l2": "per-iteration working set ~0.4 GB > 129 MB L2 (no flush needed)"},
        "phi_phiH_vis_per_s": round(vis_per_s, 1),
        "phi_phiH": {"ms": round(pair_ms, 4), "bytes": pair_bytes, "achieved_gbs": pair_gbs,
                     "frac_of_hbm_peak": {k: round(v / hbm, 4) for k, v in pair_gbs.items()}},
        "plain_fp64_gpu_iters_per_s": None if plain is None else round(plain, 3),
        "precision_fp32_vs_fp64": precision,
        "autotuned": ({"tile": tile, "chunk": chunk, "phi_phiH_ms": round(tune_ms, 4)} if tune_ms is not None
                      else {"tile": tile, "chunk": chunk, "fixed": True}),
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": round(achieved, 1), "peak": hbm,
                     "unit": "GB/s", "frac": round(achieved / hbm, 4),
                     "traffic": MEASURED_TRAFFIC.get(dom) if args.workload == WORKLOAD else None,
                     "peak_source": peak_kind, "bytes_per_launch": bytes_launch,
                     "ms_per_launch": round(dom_ms / dom_n, 4)},
        "kernels": per_kernel,
        "gpu_launches": int(launches),
        "clocks": clk.summary(),
        "e2e": e2e,
        "solver": {"objective": res.stats["objective"], "residual_over_eps": res.stats["residual"] / eps,
                   "nu": nu, "gamma": gamma, "op_device_bytes": info["device_bytes"], "work_items": info["n_items"]},
        "cpu_baseline": cpu,
        "batch_16x20": batch,
        "serving_12": serving,
    }
    if rank == 0:
        print(json.dumps(out), flush=True)
    if pg:
        pg.destroy_process_group()


# ----------------------------------------------------------------- oracle timing
def _oracle_setup(name, seed_offset=0):
    """The oracle's operator, dictionary and a measured problem of the named
    workload (same synthetic inputs as the GPU arm); build time untimed."""
    import numpy as np

    from oracle import sdmm as osdmm
    from oracle import simulate
    from oracle.nufft import NUFFT
    from paper_1406_0359_gb300 import synth

    w = synth.WORKLOADS[name]
    seed = w.seed + seed_offset
    uv = synth.uv_coverage(w.M, w.n, seed)
    x = synth.sky(w.n, seed, w.n_blobs, w.n_points)
    t = time.perf_counter()
    op = NUFFT(uv, w.n)
    build = time.perf_counter() - t
    a, b = synth.noise_draws(w.M, seed)
    y, sigma = simulate.add_noise(op.phi(x), w.isnr_db, a, b)
    psi = osdmm.SaraDictionary(w.levels)
    nu = 1.0 / math.sqrt(osdmm.operator_norm_sq(op, 3))  # any nu > 0 leaves problem (3) unchanged
    gamma = osdmm.default_gamma(op, psi, y, nu)
    return dict(w=w, op=op, psi=psi, x=x, y=y, eps=simulate.epsilon(sigma, w.M), nu=nu, gamma=gamma,
                build_s=build, weights=np.ones((9, w.n, w.n)))


def _oracle_iteration(S, st):
    """One real oracle SDMM iteration (Algorithm 1 steps 5-10, 10 CG steps), timed."""
    from oracle import sdmm as osdmm

    w = S["w"]
    t = time.perf_counter()
    osdmm.sdmm_iteration(st, S["op"], S["psi"], S["y"], S["eps"], S["gamma"], S["weights"], w.cg_iters, S["nu"])
    return time.perf_counter() - t


def _oracle_threads() -> str:
    return (f"scipy.fft on all {os.cpu_count()} host cores (workers=-1); sparse gridding/degridding and "
            f"elementwise NumPy single-threaded")


def cpu_baseline(name, gpu=None):
    """The oracle leg of the GPU arm: ONE real oracle SDMM iteration of the
    bench workload timed on the host cores, the extrapolation from one
    Phi + Phi^H pair beside it as a labelled cross-check, and -- when the GPU
    path's FP32 outputs for the same sky are given (gpu: phi, phi_adj_phi,
    psi_h) -- their relative L2 errors against the oracle's."""
    import numpy as np

    from oracle import sara as osara
    from oracle import sdmm as osdmm

    S = _oracle_setup(name)
    op, x, L = S["op"], S["x"], S["w"].levels
    st = osdmm.sdmm_init(op, S["psi"], np.zeros_like(x), S["nu"])
    it_s = _oracle_iteration(S, st)
    t = time.perf_counter()
    yx = op.phi(x)
    gx = op.phi_adj_real(yx)
    pair = time.perf_counter() - t
    t = time.perf_counter()
    cx = osara.analysis(x, L)
    osara.synthesis(cx, L)
    psi = time.perf_counter() - t
    out = {"value": round(1.0 / it_s, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
           "sample": f"one full oracle SDMM iteration of the bench workload ({w_iter(S)}), {it_s:.1f} s; "
                     f"{_oracle_threads()}; operator build {S['build_s']:.1f} s untimed",
           "extrapolated_cross_check": {"iters_per_s": round(1.0 / (12 * pair + psi), 5),
                                        "from": f"12 Phi+Phi^H pairs ({pair:.2f} s each) + one Psi^H+Psi ({psi:.2f} s)"}}
    if gpu is not None:
        outs = {"phi": yx, "phi_adj_phi": gx, "psi_h": cx}
        out["fp32_vs_oracle"] = {k: float(np.linalg.norm(gpu[k] - outs[k]) / np.linalg.norm(outs[k]))
                                 for k in ("phi", "phi_adj_phi", "psi_h")}
    return out


def w_iter(S) -> str:
    w = S["w"]
    return f"{w.cg_iters} CG steps, l1, positivity and l2-ball blocks"


def run_reference(args, ws, rank):
    """The reference arm: the FP64 oracle on the host cores, each timed step
    one real SDMM iteration of the bench workload.  Iterations run until
    `steps` are timed or the time cap is reached; `steps` reports how many
    were timed (one iteration takes tens of seconds on the CPU)."""
    if rank != 0:
        return
    import numpy as np

    from oracle import sdmm as osdmm
    from paper_1406_0359_gb300 import synth

    cap_s = float(os.environ.get("PURIFY_REFERENCE_SECONDS", "120"))
    S = _oracle_setup(args.workload)
    st = osdmm.sdmm_init(S["op"], S["psi"], np.zeros_like(S["x"]), S["nu"])
    times = []
    while len(times) < args.steps and sum(times) < cap_s:
        times.append(_oracle_iteration(S, st))
    total = sum(times)
    value = len(times) / total
    w = synth.WORKLOADS[args.workload]
    sample = (f"{len(times)} real oracle SDMM iterations of the bench workload from x = 0 ({w_iter(S)}), "
              f"{total:.1f} s in all (cap {cap_s:.0f} s, {args.steps} requested); {_oracle_threads()}; "
              f"operator build {S['build_s']:.1f} s and set-up untimed, no warm-up iteration")
    out = {"metric": METRIC, "value": round(value, 5), "unit": UNIT, "n_gpus": ws, "steps": len(times),
           "steps_requested": args.steps, "warmup": 0, "warmup_requested": args.warmup,
           "ms_per_step": round(total / len(times) * 1e3, 1), "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": {"workload": workload_string(args.workload, w)},
           "cpu_baseline": {"value": round(value, 5), "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": round(value, 5), "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- systems patterns
def _make_request(n, M, seed, dev):
    """Seeded sky, uv and noisy visibilities (y from this library's own Phi)."""
    import numpy as np
    import torch

    from paper_1406_0359_gb300 import synth
    from paper_1406_0359_gb300.binding import Operator

    uv = synth.uv_coverage(M, n, seed)
    x = synth.sky(n, seed, 3 + n // 128, 10 + n // 16)
    op = Operator(torch.as_tensor(uv, device=dev), n, 3, "fp32")
    y0 = op.phi(torch.as_tensor(x, dtype=torch.float32, device=dev)).cpu().numpy().astype(np.complex128)
    op.close()
    a, b = synth.noise_draws(M, seed)
    sigma = float(np.linalg.norm(y0)) / math.sqrt(M) * 10 ** (-1.5)
    y = y0 + sigma / math.sqrt(2) * (a + 1j * b)
    return dict(n=n, M=M, uv=uv, y=y, x=x, eps=sigma * math.sqrt(M + 2 * math.sqrt(M)))


def _snr_db(x, xh):
    import numpy as np

    return float(20 * np.log10(np.linalg.norm(x) / np.linalg.norm(np.asarray(x) - np.asarray(xh, dtype=np.float64))))


def _drain(srv, ids, arrivals=None, reqs=None, params=None):
    """Drive scheduling rounds until every request is done; with `arrivals`
    (seconds from start) requests are submitted (with `params`) as their time
    comes."""
    t0 = time.perf_counter()
    pending = list(range(len(arrivals))) if arrivals is not None else []
    while True:
        now = time.perf_counter() - t0
        while pending and arrivals[pending[0]] <= now:
            k = pending.pop(0)
            r = reqs[k]
            ids[k] = srv.submit(r["uv"], r["y"], r["n"], 3, r["eps"], **params)
        a, q = srv.step()
        if a == 0 and q == 0:
            if not pending:
                break
            time.sleep(max(0.0, min(0.002, arrivals[pending[0]] - (time.perf_counter() - t0))))
    wall = time.perf_counter() - t0
    res = [srv.result(i) for i in ids]
    return wall, res


def batch_study(count, iters, seed=4, server_arm=False, plain_arm=True):
    """`count` uneven instances (images 128/256/512 square, M uniform in
    [0.5N, 3N], seeded skies and coverages): the batched solver
    (purify_batch_solve: one launch per pass per image side, one graph per
    iteration) against the same instances solved one at a time in FP32 and by
    the plain FP64 GPU solver (no graph replay), each with `iters` SDMM
    iterations.  nu and gamma are taken once per instance and given to every
    arm; operators are built before timing.  Tile/chunk per image side from
    the autotuner."""
    import numpy as np
    import torch

    from paper_1406_0359_gb300.binding import Operator, Server, batch_solve, purify_autotune

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.choice([128, 256, 512]))
        M = int(rng.uniform(0.5, 3.0) * n * n)
        reqs.append(_make_request(n, M, seed + i, dev))
    tuned = {}
    for n in sorted({r["n"] for r in reqs}):
        r = next(q for q in reqs if q["n"] == n)
        tuned[n] = purify_autotune(torch.as_tensor(r["uv"], device=dev), n, 3)

    def ops_for(prec):
        return [Operator(torch.as_tensor(r["uv"], device=dev), r["n"], 3, prec, tile=tuned[r["n"]][0],
                         chunk=tuned[r["n"]][1]) for r in reqs]

    ops = ops_for("fp32")
    ys = [torch.as_tensor(r["y"], dtype=torch.complex64, device=dev) for r in reqs]
    eps = [r["eps"] for r in reqs]
    # nu, gamma by the library's rules, once per instance (also builds each CG operator)
    first = batch_solve(ops, ys, eps, t_max=1, cg_iters=1)
    nus, gammas = [r.stats["nu"] for r in first], [r.stats["gamma"] for r in first]
    kw = dict(t_max=iters, cg_iters=10)
    batch_solve(ops, ys, eps, nu=nus, gamma=gammas, **kw)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    res_b = batch_solve(ops, ys, eps, nu=nus, gamma=gammas, **kw)
    torch.cuda.synchronize()
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    res_s = [op.solve(y, e, nu=nu, gamma=g, **kw) for op, y, e, nu, g in zip(ops, ys, eps, nus, gammas)]
    torch.cuda.synchronize()
    t_s = time.perf_counter() - t0
    out = {"instances": count, "iterations_per_solve": iters,
           "batched_solves_per_s": round(count / t_b, 3), "sequential_fp32_solves_per_s": round(count / t_s, 3),
           "speedup_vs_sequential_fp32": round(t_s / t_b, 3),
           "max_rel_diff_batched_vs_alone": max(float(torch.linalg.vector_norm(a.x - b.x) / torch.linalg.vector_norm(b.x))
                                                for a, b in zip(res_b, res_s)),
           "autotuned": {str(k): {"tile": v[0], "chunk": v[1]} for k, v in tuned.items()}}
    xb = [r.x.cpu().numpy().astype(np.float64) for r in res_b]
    out["snr_db_mean"] = round(float(np.mean([_snr_db(r["x"], x) for r, x in zip(reqs, xb)])), 4)
    for o in ops:
        o.close()
    if plain_arm:
        ops64 = ops_for("fp64")
        ys64 = [y.to(torch.complex128) for y in ys]
        ops64[0].solve(ys64[0], eps[0], nu=nus[0], gamma=gammas[0], t_max=1, cg_iters=1, use_graph=False)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res_p = [op.solve(y, e, nu=nu, gamma=g, use_graph=False, **kw)
                 for op, y, e, nu, g in zip(ops64, ys64, eps, nus, gammas)]
        torch.cuda.synchronize()
        t_p = time.perf_counter() - t0
        xp = [r.x.cpu().numpy() for r in res_p]
        snr_p = [_snr_db(r["x"], x) for r, x in zip(reqs, xp)]
        out.update({"plain_fp64_solves_per_s": round(count / t_p, 3), "speedup_vs_plain_fp64": round(t_p / t_b, 3),
                    "max_rel_diff_vs_plain_fp64": max(float(np.linalg.norm(a - b) / np.linalg.norm(b))
                                                      for a, b in zip(xb, xp)),
                    "snr_db_mean_plain_fp64": round(float(np.mean(snr_p)), 4),
                    "max_abs_snr_diff_db": round(float(np.max(np.abs(np.array(
                        [_snr_db(r["x"], x) for r, x in zip(reqs, xb)]) - np.array(snr_p)))), 6)})
        for o in ops64:
            o.close()
    if server_arm:  # the request server with every instance admitted at once
        for batching, key in ((False, "server_all_admitted_solves_per_s"),
                              (True, "server_all_admitted_iteration_batched_solves_per_s")):
            srv = Server(int(150e9), count)
            srv.set_batching(batching)
            for n, (tile, chunk, _) in tuned.items():
                srv.set_options(n, tile, chunk)
            ids = [srv.submit(r["uv"], r["y"], r["n"], 3, r["eps"], nu=nu, gamma=g, **kw)
                   for r, nu, g in zip(reqs, nus, gammas)]
            wall, _ = _drain(srv, ids)
            if batching:
                out["server_batched_iteration_share"] = round(srv.counts()[0] / max(1, sum(srv.counts())), 4)
            srv.close()
            out[key] = round(count / wall, 3)
    return out


def run_batch(args):
    """C4: 64 uneven instances through the batched solver against one at a
    time (FP32 graph replay; plain FP64), and the request server's form."""
    from paper_1406_0359_gb300 import build as _build

    _build.build()
    res = batch_study(args.batch_size, args.batch_iters, server_arm=True)
    line = {"metric": f"batched SARA-SDMM solves/s, {args.batch_size} uneven instances (128..512 square, "
                      "M in [0.5N, 3N])", "value": res["batched_solves_per_s"], "unit": "solves/s",
            "higher_is_better": True, "dtype": "f32 (compensated reductions, FP64 finals)", "data": "synthetic",
            "config": {"workload": f"{args.batch_size} independent solves, seeds 4+i",
                       "mode": "purify_batch_solve: one launch per pass per image side, one graph per iteration"}}
    line.update(res)
    print(json.dumps(line), flush=True)


def serving_summary(count=12, seed=7, rate_mult=2.0):
    """Reduced form of the serving benchmark for the default bench line:
    `count` requests (images 128^2-512^2, M log-uniform in [16K, 256K], SDMM
    to xi = 1e-4 or 100 iterations), one at a time through the server, then
    as Poisson arrivals at `rate_mult` times that rate with 16 slots:
    solves/s, p50 / p99 latency and the worst difference from the one-at-a-time
    results."""
    import numpy as np
    import torch

    from paper_1406_0359_gb300.binding import Server

    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(count):
        n = int(rng.choice([128, 256, 512], p=[0.4, 0.35, 0.25]))
        M = int(np.exp(rng.uniform(np.log(16384), np.log(1 << 18))))
        reqs.append(_make_request(n, M, 900 + i, dev))
    params = dict(t_max=100, cg_iters=10, xi=1e-4)
    srv = Server(int(150e9), 1)
    ids = [srv.submit(r["uv"], r["y"], r["n"], 3, r["eps"], **params) for r in reqs]
    seq_wall, seq_res = _drain(srv, ids)
    srv.close()
    lam = rate_mult * count / seq_wall
    arr = np.cumsum(np.random.default_rng(seed + 1).exponential(1.0 / lam, count))
    srv = Server(int(150e9), 16)
    ids = [None] * count
    wall, res = _drain(srv, ids, list(arr), reqs, params)
    srv.close()
    srv = Server(int(150e9), 16)
    srv.set_batching(True)
    wall_b, _ = _drain(srv, [None] * count, list(arr), reqs, params)
    cnt = srv.counts()
    srv.close()
    lat = np.array([r[2] for r in res])
    return {"requests": count, "one_at_a_time_solves_per_s": round(count / seq_wall, 3),
            "offered_rps": round(lam, 3), "solves_per_s": round(count / wall, 3),
            "iteration_batched_solves_per_s": round(count / wall_b, 3),
            "iteration_batched_share": round(cnt[0] / max(1, sum(cnt)), 4),
            "p50_s": round(float(np.percentile(lat, 50)), 4), "p99_s": round(float(np.percentile(lat, 99)), 4),
            "max_rel_diff_vs_alone": max(float(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0]))
                                         for a, b in zip(res, seq_res)),
            "note": "reduced form of bench.py --serving: images 128^2-512^2, M 16K-256K, xi = 1e-4 or 100 iterations"}


def run_serving(args):
    """Poisson arrivals of mixed-size solve requests (images 128^2 to 2048^2,
    M log-uniform in [16K, 16M], SDMM to xi = 1e-4 or 300 iterations) through the
    continuous-batching server (150 GB budget, 16 slots), at rates relative to
    the one-at-a-time throughput; p50/p99 latency and solves/s per rate.  The
    2048^2 requests use the NUFFT form of the CG operator (the convolution
    form needs n <= 1024)."""
    import numpy as np
    import torch

    from paper_1406_0359_gb300 import build as _build
    from paper_1406_0359_gb300.binding import Server

    _build.build()
    dev = torch.device("cuda", 0)
    rng = np.random.default_rng(5)
    reqs = []
    for i in range(args.serve_requests):
        n = int(rng.choice([128, 256, 512, 1024, 2048], p=[0.3, 0.27, 0.23, 0.13, 0.07]))
        M = int(np.exp(rng.uniform(np.log(16384), np.log(16 << 20))))
        reqs.append(_make_request(n, M, 500 + i, dev))
    params = dict(t_max=300, cg_iters=10, xi=1e-4)
    srv = Server(int(150e9), 1)
    ids = [srv.submit(r["uv"], r["y"], r["n"], 3, r["eps"], **params) for r in reqs]
    seq_wall, seq_res = _drain(srv, ids)
    srv.close()
    seq_rate = len(reqs) / seq_wall
    # the plain GPU solver (FP64, no graph replay), one request at a time
    srv = Server(int(150e9), 1)
    ids = [srv.submit(r["uv"], r["y"], r["n"], 3, r["eps"], precision="fp64", use_graph=0, **params) for r in reqs]
    p64_wall, p64_res = _drain(srv, ids)
    srv.close()
    rates = []
    for mult in (0.5, 1.0, 2.0, 4.0):
        lam = mult * seq_rate
        arr = np.cumsum(np.random.default_rng(int(mult * 10)).exponential(1.0 / lam, len(reqs)))
        srv = Server(int(150e9), 16)
        ids = [None] * len(reqs)
        wall, res = _drain(srv, ids, list(arr), reqs, params)
        srv.close()
        lat = np.array([r[2] for r in res])
        worst = max(float(np.linalg.norm(a[0] - b[0]) / np.linalg.norm(b[0])) for a, b in zip(res, seq_res))
        rates.append({"offered_rps": round(lam, 3), "solves_per_s": round(len(reqs) / wall, 3),
                      "p50_s": round(float(np.percentile(lat, 50)), 4), "p99_s": round(float(np.percentile(lat, 99)), 4),
                      "max_rel_diff_vs_alone": worst})
    best = max(rates, key=lambda r: r["solves_per_s"])
    snr_s = [_snr_db(r["x"], x[0]) for r, x in zip(reqs, seq_res)]
    snr_p = [_snr_db(r["x"], x[0]) for r, x in zip(reqs, p64_res)]
    line = {"metric": "serving solves/s and p50/p99 latency (continuous batching)", "value": best["solves_per_s"],
            "unit": "solves/s", "higher_is_better": True, "one_at_a_time_solves_per_s": round(seq_rate, 3),
            "plain_fp64_one_at_a_time_solves_per_s": round(len(reqs) / p64_wall, 3),
            "snr_db_mean": round(float(np.mean(snr_s)), 4), "snr_db_mean_plain_fp64": round(float(np.mean(snr_p)), 4),
            "max_abs_snr_diff_db": round(float(np.max(np.abs(np.array(snr_s) - np.array(snr_p)))), 6),
            "rates": rates, "requests": len(reqs), "dtype": "f32 (compensated reductions, FP64 finals)",
            "data": "synthetic",
            "config": {"workload": "Poisson arrivals, images 128..2048, M log-uniform 16K..16M, xi=1e-4 or 300 it.",
                       "budget_gb": 150, "slots": 16}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--workload", default=WORKLOAD)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-batch-summary", action="store_true")
    ap.add_argument("--tile", type=int, default=0, help="with --chunk: skip the autotuner (8 or 16)")
    ap.add_argument("--chunk", type=int, default=0, help="with --tile: visibilities per work item")
    ap.add_argument("--batch", action="store_true", help="64 uneven instances: batched vs one at a time")
    ap.add_argument("--batch-size", type=int, default=64)
    ap.add_argument("--batch-iters", type=int, default=50)
    ap.add_argument("--serving", action="store_true", help="Poisson-arrival serving benchmark")
    ap.add_argument("--serve-requests", type=int, default=40)
    args = ap.parse_args()
    if args.batch:
        run_batch(args)
        return
    if args.serving:
        run_serving(args)
        return
    if args.warmup < 3:
        args.warmup = 3
    ws, rank, local = dist_info()
    if args.impl == "reference":
        run_reference(args, ws, rank)
    else:
        run_ours(args, ws, rank, local)


if __name__ == "__main__":
    main()
