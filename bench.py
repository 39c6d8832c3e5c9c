"""Benchmark of the UoI_LASSO hot path on one GB300 (or N replicas under torchrun).

Default workload: UoI_LASSO at scale -- X 50000 x 2000 with Toeplitz(0.5) rows,
5 % nonzero beta, SNR 5, B1 = q = B2 = 48 -- in the mixed-precision form.  One
step = one full fit (selection: 48 x 48 LASSO-ADMM columns, intersection;
estimation: 48 bootstraps x 48 support OLS fits, held-out loss argmin,
median bagging).  The design (800 MB) is larger than L2, and it is resident
in HBM when the device-timed region starts.

Prints one JSON line (rank 0).  --impl reference times the FP64 CPU oracle on
a bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "UoI fits/s & ADMM LASSO solves/s vs plain FP64 GPU form at ≤1e-5 coef error"
DTYPE_MIXED = ("mixed: Gram bf16 2-piece/3 products, inverse + x-update fp16 2-piece/3 products, "
               "f32 accumulation and ADMM state, f64 OLS refinement and bagging")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default 20 on the workloads whose fit takes well under a "
                         "second, 5 on the VAR p = 1000 workload and in the reference arm)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--warm", default="none", choices=["none", "path", "learned"],
                    help="ADMM start: cold lambda batch, path warm start, or the learned start (a network "
                         "trained first, outside the timed region, on problems with disjoint seeds)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--fp64-steps", type=int, default=None,
                    help="timed fits of the plain FP64 GPU form on the same inputs (mixed runs only; "
                         "default 2 on the 50000 x 2000 workload, 0 elsewhere; 0 skips the baseline "
                         "and the coefficient-error comparison)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # size overrides for profiling captures on a small case (the line is then not a
    # bench line: config.overrides says so)
    ap.add_argument("--B1", type=int)
    ap.add_argument("--B2", type=int)
    ap.add_argument("--q", type=int)
    ap.add_argument("--rows", type=int, help="keep only the first ROWS rows of the design")
    ap.add_argument("--streams", type=int, default=0,
                    help="batched workload: 0 = grouped ADMM over all problems, N > 0 = N worker streams")
    ap.add_argument("--order", type=int, default=1, help="VAR workloads: lag order d of the design")
    ap.add_argument("--intercept", type=int, default=0, choices=[0, 1],
                    help="VAR workloads: fit the unpenalised intercept mu")
    ap.add_argument("--block-mode", default="fixed", choices=["fixed", "moving"],
                    help="selection blocks of the block bootstrap: non-overlapping or moving")
    ap.add_argument("--split", default="per_bootstrap", choices=["per_bootstrap", "fixed"],
                    help="estimation split: a fresh reshuffle per bootstrap or one for all")
    ap.add_argument("--bagging", default=None, choices=["median", "mean"],
                    help="bagging of the chosen estimates (default: the workload's)")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi polled every 50 ms in a child process; each line is stamped with
    the host's monotonic clock when it arrives, so that the summary keeps only the
    samples taken inside the timed region (mark_start / mark_stop).  start() waits
    for the first sample, so that sampling is running before the region opens."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 50

    def __init__(self, gpu_index, cmd=None):
        self.gpu = gpu_index
        self.cmd = cmd or ["nvidia-smi", "-i", str(gpu_index), f"--query-gpu={self.FIELDS}",
                           "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)]
        self.proc = None
        self.lines = []                                  # (host time, line)
        self.t0 = self.t1 = None

    def start(self, ready_timeout=5.0):
        try:
            self.proc = subprocess.Popen(self.cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
            return
        end = time.monotonic() + ready_timeout
        while not self.lines and time.monotonic() < end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.monotonic(), ln.strip()))

    def mark_start(self):
        self.t0 = time.monotonic()

    def mark_stop(self):
        self.t1 = time.monotonic()

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.t.join(timeout=5)
        return self.summary()

    def summary(self):
        lines = list(self.lines)
        if self.t0 is not None and self.t1 is not None:
            # a line arrives up to one period after the sample it reports
            inside = [(t, ln) for t, ln in lines if self.t0 <= t <= self.t1 + self.PERIOD_MS / 1e3]
            lines = inside or lines
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for _, ln in lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# workload
# ----------------------------------------------------------------------------
def workload(wid, order=1):
    from paper_1808_06992_gb300 import synth
    w = synth.WORKLOADS[wid]
    d = synth.workload_data(wid)
    if w.kind == "lasso":
        X, Y = d.X, d.y.reshape(-1, 1)
    elif w.kind == "var":
        # lagged design of a VAR(order): response X_t, regressors X_{t-1} .. X_{t-order}
        S = d.series
        N = S.shape[0]
        X = np.concatenate([S[order - j:N - j] for j in range(1, order + 1)], axis=1)
        Y = S[order:]
    else:
        raise ValueError("the batched workload is timed by bench_batch")
    return w, np.ascontiguousarray(X), np.ascontiguousarray(Y)


def fit_kwargs(w, args):
    from paper_1808_06992_gb300 import native
    bag = w.bagging if args.bagging is None else (1 if args.bagging == "mean" else 0)
    warm = {"none": native.WARM_NONE, "path": native.WARM_PATH, "learned": native.WARM_LEARNED}[args.warm]
    kw = dict(B1=args.B1 or w.B1, B2=args.B2 or w.B2, q=args.q or w.q, block_len=w.block_len,
              bagging=bag, block_mode=1 if args.block_mode == "moving" else 0,
              split_mode=native.SPLIT_FIXED if args.split == "fixed" else native.SPLIT_PER_BOOTSTRAP,
              precision=native.PREC_MIXED if args.precision == "mixed" else native.PREC_FP64,
              warm_start=warm, intercept=args.intercept if w.kind == "var" else 0)
    if args.warm == "learned":
        kw["mlp_weights_path"] = args.mlp_weights
    return kw


def train_warm_start(w, args):
    """Trains the learned start's network before the timed region on rows from the
    method's own path-warm solutions of problems shaped like the workload (seeds
    disjoint from the workload's); returns a description for the bench line."""
    import tempfile

    from paper_1808_06992_gb300 import warm_start
    t0 = time.time()
    args.mlp_weights = os.path.join(tempfile.mkdtemp(prefix="uoi_ws_"), "ws.bin")
    prm = w.params
    if w.kind == "var":
        p = min(int(prm["p"]), 200)
        F, T = warm_start.var_training_rows(p, 2000, max(prm["density"], 0.05), prm["spectral_radius"],
                                            w.block_len, args.q or w.q)
        what = f"VAR(1) p={p}, 2 series"
    else:
        F, T = warm_start.lasso_training_rows(200, 50, 10, args.q or w.q)
        what = "24 LASSO problems 200 x 50"
    L0, L1 = warm_start.train(F, T, args.mlp_weights)
    return {"rows": int(F.shape[0]), "problems": what, "loss_initial": L0, "loss_final": L1,
            "seconds": time.time() - t0}


def traffic_per_launch(kernel, applies=True):
    """DRAM bytes per launch from the committed ncu capture, if the kernel's source
    still matches the hash recorded with it and the run is the workload the figure
    was scaled to (else None)."""
    import hashlib
    if not applies:
        return None
    path = os.path.join(ROOT, "profiles", "traffic.txt")
    src = {"k_gram_tc": "gram_tc.cu", "k_stream_gemm": "admm.cu", "k_xupdate_tc": "xupdate_tc.cu"}[kernel]
    try:
        with open(os.path.join(ROOT, "paper_1808_06992_gb300", "csrc", src), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()[:16]
        with open(path) as f:
            for ln in f:
                fields = dict(kv.split("=", 1) for kv in ln.split() if "=" in kv)
                if fields.get("kernel") == kernel and fields.get("source_sha") == sha:
                    return float(fields["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        pass
    return None


def algorithmic_gram_flops(m, p, r, rows):
    """2 * rows * (p(p+1)/2 + p r): symmetric half of X^T W X plus X^T W Y."""
    return 2.0 * rows * (p * (p + 1) / 2 + p * r)


# ----------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on a bounded sample of the workload
# ----------------------------------------------------------------------------
def host_cores():
    """Threads this process may run on, and the host's logical CPU count from /proc/cpuinfo."""
    try:
        avail = len(os.sched_getaffinity(0))
    except AttributeError:
        avail = os.cpu_count() or 1
    listed = 0
    try:
        with open("/proc/cpuinfo") as f:
            listed = sum(1 for ln in f if ln.startswith("processor"))
    except OSError:
        pass
    return avail, listed or avail


def cpu_sample(w, X, Y, threads=1, support_size=100, admm_cols=4):
    """Times oracle stages and extrapolates to one full fit on ``threads`` cores.

    Each of ``threads`` concurrent workers times the stages of its own selection
    bootstrap k (the oracle's OpenMP loop runs bootstraps in parallel, one per
    thread): the weighted Gram over a row sample (per multiply-add rate), one
    Cholesky of order min(p, 1000) scaled by p^3, path-warm ADMM columns over a
    sample of ``admm_cols`` lambdas spread over the grid, and one OLS on a support of
    ``support_size`` features.  The
    fit time is rebuilt from the workload's operation counts, with B1 and B2
    bootstraps spread over the threads (ceil(B / threads) rounds each).
    Returns (fits_per_s, solves_per_s, description)."""
    import concurrent.futures as cf

    import oracle
    m, p = X.shape
    r = Y.shape[1]
    t_all = time.time()
    rows = min(m, max(200, int(1.0e9 / (p * (p + r)))))
    lam = oracle.lambda_grid(oracle.lambda_max(X, Y), w.q)
    jsel = list(range(0, w.q, max(1, w.q // admm_cols)))[:admm_cols]
    pc = min(p, 1000)
    s_ols = min(p, support_size)
    bits = np.zeros((p + 63) // 64, dtype=np.uint64)
    for i in range(s_ols):
        bits[i // 64] |= np.uint64(1) << np.uint64(i % 64)

    def stages(k):
        w0 = oracle.selection_weights(m, w.block_len, 0, 0, k)
        ws = w0.copy()
        ws[rows:] = 0
        nz_rows = int(np.count_nonzero(ws))
        t = time.time()
        G, B = oracle.weighted_moments(X, Y, ws)
        t_fma = (time.time() - t) / max(nz_rows * p * (p + r), 1)
        nk = float(ws.sum())
        A = G / nk + np.eye(p)
        t = time.time()
        L_c, _ = oracle.cholesky(A[:pc, :pc])
        t_chol = (time.time() - t) * (p / pc) ** 3
        L, _ = oracle.cholesky(A) if pc < p else (L_c, 0)
        t = time.time()
        its = 0
        z = np.zeros(p)
        u = np.zeros(p)
        for j in jsel:
            res = oracle.admm_column(L, B[:, 0] / nk, lam[j], z0=z, u0=u)
            z, u = res["z"], res["u"]
            its += res["iters"]
        t_admm_col = (time.time() - t) / len(jsel)
        t = time.time()
        oracle.ols_support(G, B[:, 0], bits)
        t_ols = time.time() - t
        return dict(t_fma=t_fma, t_chol=t_chol, t_admm_col=t_admm_col, t_ols=t_ols, its=its,
                    nz_rows=nz_rows, nz_sel=int(np.count_nonzero(w0)))

    with cf.ThreadPoolExecutor(max_workers=threads) as ex:
        res = list(ex.map(stages, range(threads)))
    mean = {key: float(np.mean([rr[key] for rr in res])) for key in res[0]}
    n_eval = m - int(np.floor(0.8 * m))
    t_loss = n_eval * p * mean["t_fma"]
    train_rows = int(0.8 * m * (1 - np.exp(-1)))
    n_cols = w.B1 * w.q * r
    t_sel_boot = mean["nz_sel"] * p * (p + r) * mean["t_fma"] + mean["t_chol"] + w.q * r * mean["t_admm_col"]
    t_est_boot = train_rows * p * (p + r) * mean["t_fma"] + w.q * r * (mean["t_ols"] + t_loss)
    rounds1 = -(-w.B1 // threads)
    rounds2 = -(-w.B2 // threads)
    t_fit = rounds1 * t_sel_boot + rounds2 * t_est_boot
    desc = (f"FP64 oracle on {threads} thread(s), each timing the stages of its own selection bootstrap: "
            f"Gram over {int(mean['nz_rows'])} of {m} rows, one {pc}x{pc} Cholesky scaled by (p/{pc})^3, "
            f"{len(jsel)} path-warm ADMM columns ({int(mean['its'])} iterations), one OLS on {s_ols} features; "
            f"extrapolated by operation counts to B1={w.B1}, q={w.q}, B2={w.B2} with ceil(B/{threads}) "
            f"bootstrap rounds per thread ({t_fit:.0f} s per fit); sample took {time.time() - t_all:.1f} s")
    return 1.0 / t_fit, n_cols / t_fit, desc


def max_over_ranks(value, dist, device="cuda"):
    """The largest of every rank's value (the value itself on one rank): the
    step time a multi-rank run reports is the slowest rank's."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_1808_06992_gb300 import synth
    w, X, Y = workload(args.workload, args.order if synth.WORKLOADS[args.workload].kind == "var" else 1)
    import oracle
    oracle.build_oracle()
    threads, listed = host_cores()
    vals, secs = [], []
    desc = ""
    # the whole run stays within a few minutes: warm-up steps sample one ADMM column,
    # timed steps four (two when there are more than 8 of them)
    cols = 4 if args.steps <= 8 else 2
    for i in range(args.warmup + args.steps):
        t0 = time.time()
        fps, sps, d = cpu_sample(w, X, Y, threads=threads, admm_cols=1 if i < args.warmup else cols)
        if i >= args.warmup:
            vals.append(fps)
            secs.append(time.time() - t0)
            desc = d
    v = float(np.mean(vals))
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "fits/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / v,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name},
            "cpu_baseline": {"value": v, "unit": "fits/s", "cores": threads, "host_cpus": listed,
                             "kind": "oracle", "sample": desc,
                             "sample_wall_s_per_step": float(np.mean(secs))},
            "e2e": {"value": v, "unit": "fits/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
def main():
    args = parse()
    if args.steps is None:
        args.steps = 5 if (args.impl == "reference" or args.workload == 5) else 20
    if args.fp64_steps is None:
        args.fp64_steps = 2 if args.workload == 2 else 0
    if args.impl == "reference":
        return run_reference(args)
    import torch
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1808_06992_gb300 import native, synth
    native.lib()
    if synth.WORKLOADS[args.workload].kind == "batch":
        return bench_batch(args, torch, rank, world, local, dist)
    w, X, Y = workload(args.workload, args.order if synth.WORKLOADS[args.workload].kind == "var" else 1)
    if args.rows:
        X, Y = np.ascontiguousarray(X[:args.rows]), np.ascontiguousarray(Y[:args.rows])
    m, p = X.shape
    r = Y.shape[1]
    ws_train = train_warm_start(w, args) if args.warm == "learned" else None
    kw = fit_kwargs(w, args)
    overrides = {k: getattr(args, k) for k in ("B1", "B2", "q", "rows") if getattr(args, k)}
    if w.kind == "var" and (args.order != 1 or args.intercept):
        overrides.update(order=args.order, intercept=args.intercept)
    for k, dflt in (("block_mode", "fixed"), ("split", "per_bootstrap")):
        if getattr(args, k) != dflt:
            overrides[k] = getattr(args, k)
    if args.bagging is not None:
        overrides["bagging"] = args.bagging
    Xd = torch.from_numpy(X).cuda()
    Yd = torch.from_numpy(Y).cuda()
    stream = torch.cuda.current_stream().cuda_stream

    def step():
        return native.uoi_fit_traced(Xd, Yd, trace=False, stream=stream, **kw)

    for _ in range(args.warmup):
        out = step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark_start()
    ev0.record()
    diags = []
    for _ in range(args.steps):
        out = step()
        diags.append(out["diag"])
    ev1.record()
    torch.cuda.synchronize()
    sampler.mark_stop()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    ms_step = ms / args.steps
    fits_s = world * args.steps / (ms / 1e3)
    cols = w.B1 * w.q * r
    # Per-kernel live timing: the library records CUDA events on the launch stream
    # around every tensor-core Gram and x-update launch of the step and
    # reports their algorithmic work (flops of the math, not of the split products).
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    bf16 = peaks.get("bf16_tflops")
    hbm = peaks.get("hbm_gbs")
    fp64_peak = 1.25                                     # nominal GB300 FP64 (no measured figure)
    # the committed traffic figures are scaled to the default workload and form
    default_run = (not overrides and args.workload == 2 and args.precision == "mixed"
                   and args.warm == "none")
    kernels = []
    ms_g = sum(d["ms_gram_tc"] for d in diags)
    if ms_g > 0:
        fl = sum(d["flops_gram_tc"] for d in diags)
        n = sum(d["n_gram_tc"] for d in diags)
        ach = fl / (ms_g / 1e3) / 1e12
        peak = (bf16 / 3.0) if bf16 else 1900.0 / 3.0
        kernels.append({"kernel": "k_gram_tc (tensor-core Gram, split bf16 x3)", "bound": "tensor",
                        "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                        "traffic": traffic_per_launch("k_gram_tc", default_run), "launches_per_step": n / args.steps,
                        "ms_per_step": ms_g / args.steps,
                        "peak_source": ("measured bf16 burst / 3 (three bf16 products per "
                                        "FP32-accurate multiply-add)" if bf16 else "fallback 1.9 PF / 3"),
                        "tensor_pipe_frac": ach * 3.0 / (bf16 or 1900.0)})
    ms_x = sum(d["ms_xupdate"] for d in diags)
    if ms_x > 0:
        fl = sum(d["flops_xupdate"] for d in diags)
        by = sum(d["bytes_xupdate"] for d in diags)
        n = sum(d["n_xupdate"] for d in diags)
        ach = fl / (ms_x / 1e3) / 1e12
        gbs = by / (ms_x / 1e3) / 1e9
        if args.precision == "mixed":
            # tensor-core x-update: streams the three bf16 pieces of every group's
            # inverse once per iteration; the algorithmic bytes count M once in FP32
            hpeak = hbm or 6800.0
            kernels.append({"kernel": "k_xupdate_tc (ADMM x-update on tcgen05, fused z/u/norm epilogue)",
                            "bound": "hbm", "achieved": gbs, "peak": hpeak, "unit": "GB/s",
                            "frac": gbs / hpeak, "traffic": traffic_per_launch("k_xupdate_tc", default_run),
                            "launches_per_step": n / args.steps, "ms_per_step": ms_x / args.steps,
                            "tflops_algorithmic": ach,
                            "peak_source": "measured HBM copy" if hbm else "fallback 6.8 TB/s"})
        else:
            kernels.append({"kernel": "k_stream_gemm (FP64 ADMM x-update + fused epilogue)", "bound": "alu",
                            "achieved": ach, "peak": fp64_peak, "unit": "TFLOP/s", "frac": ach / fp64_peak,
                            "traffic": traffic_per_launch("k_stream_gemm", False), "launches_per_step": n / args.steps,
                            "ms_per_step": ms_x / args.steps,
                            "hbm_gbs_algorithmic": gbs,
                            "hbm_frac_algorithmic": gbs / hbm if hbm else None,
                            "peak_source": "nominal FP64 1.25 TFLOP/s"})
    kernels.sort(key=lambda k: -k["ms_per_step"])
    roofline = kernels[0] if kernels else None
    stage_ms = {k: float(np.mean([d[f"ms_{k}"] for d in diags]))
                for k in ("gram", "factor", "admm", "estimation")}
    launches = int(np.mean([d["gpu_launches"] for d in diags]))
    # end to end: host (pinned) inputs, result read back, through the public API
    e2e = None
    if args.e2e_steps > 0:
        Xh = torch.from_numpy(X).pin_memory()
        Yh = torch.from_numpy(Y).pin_memory()
        Xn, Yn = Xh.numpy(), Yh.numpy()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            res = native.uoi_fit_traced(Xn, Yn, trace=False, **kw)
            _ = float(np.asarray(res["beta"]).sum())
        t1 = time.perf_counter()
        e2e = {"value": args.e2e_steps / (t1 - t0), "unit": "fits/s",
               "h2d_bytes_per_step": int(X.nbytes + Y.nbytes), "d2h_bytes_per_step": int(r * p * 8)}
    # the metric's baseline: the plain FP64 GPU form on the same device-resident
    # inputs, and the coefficient error of the timed form against it
    base = None
    if args.precision == "mixed" and args.fp64_steps > 0:
        base = fp64_baseline(args, native, torch, Xd, Yd, kw, stream, out, fits_s, world)
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads, listed = host_cores()
        fps, sps, desc = cpu_sample(w, X, Y, threads=threads)
        fps1, sps1, desc1 = cpu_sample(w, X, Y, threads=1)
        cpu = {"value": fps, "unit": "fits/s", "cores": threads, "host_cpus": listed, "kind": "oracle",
               "sample": desc, "solves_per_s": sps,
               "single_thread": {"value": fps1, "unit": "fits/s", "cores": 1, "solves_per_s": sps1,
                                 "sample": desc1}}
    if rank == 0:
        line = {"metric": METRIC, "value": fits_s, "unit": "fits/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak",
                "vs_baseline": base["vs_fp64_gpu"] if base else None,
                "baseline": base,
                "dtype": DTYPE_MIXED if args.precision == "mixed" else "f64",
                "data": "synthetic",
                "config": {"workload": w.name, "n": m, "p": p, "r": r, "B1": w.B1, "q": w.q,
                           "B2": w.B2, "precision": args.precision, "warm_start": args.warm,
                           **({"warm_start_training": ws_train} if ws_train else {}),
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "inputs larger than L2 (X is %.0f MB)" % (X.nbytes / 1e6),
                           **({"overrides": overrides} if overrides else {})},
                "solves_per_s": fits_s * cols,
                "admm": {"iterations_per_fit": float(np.mean([d["admm_iterations"] for d in diags])),
                         "nonconverged_per_fit": float(np.mean([d["admm_nonconverged"] for d in diags])),
                         "warm_start_used": ["none", "path", "learned"][diags[-1]["warm_start_used"]]},
                "roofline": roofline, "roofline_other": kernels[1:], "stage_ms": stage_ms,
                "clocks": clocks, "gpu_launches": launches * args.steps,
                "e2e": e2e, "cpu_baseline": cpu,
                "diag": diags[-1]}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def fp64_baseline(args, native, torch, Xd, Yd, kw, stream, out_mixed, fits_mixed, world):
    """Times the plain FP64 GPU form (UOI_PREC_FP64) on the same device inputs and
    compares the bagged estimate, the family and j* of the timed mixed fit with it.
    The first (untimed) FP64 fit is traced and gives the reference values; an untimed
    traced mixed fit gives the mixed family and j* (its beta* must equal the timed
    fits' bit for bit: the fit is deterministic)."""
    kw64 = dict(kw, precision=native.PREC_FP64)
    ref = native.uoi_fit_traced(Xd, Yd, trace=True, stream=stream, **kw64)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.fp64_steps):
        native.uoi_fit_traced(Xd, Yd, trace=False, stream=stream, **kw64)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.fp64_steps
    mix = native.uoi_fit_traced(Xd, Yd, trace=True, stream=stream, **kw)
    bm = mix["beta"].double().cpu().numpy()
    bf = ref["beta"].double().cpu().numpy()
    nb = float(np.linalg.norm(bf))
    err = float(np.linalg.norm(bm - bf) / nb) if nb > 0 else float(np.linalg.norm(bm - bf))
    fm = mix["family"].cpu().numpy().view(np.uint64)
    ff = ref["family"].cpu().numpy().view(np.uint64)
    differ = int(sum(bin(int(x)).count("1") for x in np.bitwise_xor(fm, ff).ravel()))
    total = int(sum(bin(int(x)).count("1") for x in ff.ravel()))
    sm = mix["sel_beta"].cpu().numpy()
    sf = ref["sel_beta"].cpu().numpy()
    num = np.linalg.norm(sm - sf, axis=-1)
    den = np.linalg.norm(sf, axis=-1)
    sel_rel = float(np.max(np.where(den > 0, num / np.where(den > 0, den, 1.0), num)))
    fps = world * 1e3 / ms
    return {"form": "plain FP64 GPU (UOI_PREC_FP64), same device-resident inputs",
            "value": fps, "unit": "fits/s", "ms_per_step": ms, "steps": args.fp64_steps, "warmup": 1,
            "vs_fp64_gpu": fits_mixed / fps,
            "coef_rel_l2": err, "coef_tol": 1e-5, "coef_within_tol": err <= 1e-5,
            "family_bits_differ": differ, "family_bits_fp64": total,
            "jstar_identical": bool(np.array_equal(mix["est_jstar"].cpu().numpy(), ref["est_jstar"].cpu().numpy())),
            "timed_beta_identical": bool(np.array_equal(out_mixed["beta"].double().cpu().numpy(), bm)),
            "selection_max_rel_l2_vs_fp64": sel_rel,
            "fp64_stage_ms": {k: float(ref["diag"][f"ms_{k}"]) for k in ("gram", "factor", "admm", "estimation")}}


def bench_batch(args, torch, rank, world, local, dist):
    """Batched uneven problems: one step = one uoi_lasso_fit_batch call over the
    workload's independent problems; fits/s counts problems."""
    from paper_1808_06992_gb300 import native, synth
    w = synth.WORKLOADS[args.workload]
    probs = synth.workload_data(args.workload)
    kw = fit_kwargs(w, args)
    Xd = [torch.from_numpy(np.ascontiguousarray(pb.X)).cuda() for pb in probs]
    yd = [torch.from_numpy(np.ascontiguousarray(pb.y)).cuda() for pb in probs]
    count = len(probs)

    def step():
        return native.uoi_lasso_fit_batch(Xd, yd, streams=args.streams, **kw)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    sampler.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    sampler.mark_start()
    ev0.record()
    outs = []
    for _ in range(args.steps):
        outs.append(step())          # returns once every worker stream has finished
    ev1.record()
    torch.cuda.synchronize()
    sampler.mark_stop()
    if dist:
        dist.barrier()
    clocks = sampler.stop()
    ms = max_over_ranks(ev0.elapsed_time(ev1), dist)
    fits_s = world * args.steps * count / (ms / 1e3)
    diags = [o["diag"] for o in outs[-1]]
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    bf16 = peaks.get("bf16_tflops")
    hbm = peaks.get("hbm_gbs")
    kernels = []
    ms_g = sum(d["ms_gram_tc"] for d in diags)
    if ms_g > 0:
        ach = sum(d["flops_gram_tc"] for d in diags) / (ms_g / 1e3) / 1e12
        peak = (bf16 / 3.0) if bf16 else 1900.0 / 3.0
        kernels.append({"kernel": "k_gram_tc (tensor-core Gram, split bf16 x3)", "bound": "tensor",
                        "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak, "traffic": None,
                        "launches_per_step": sum(d["n_gram_tc"] for d in diags), "ms_per_step": ms_g,
                        "peak_source": "measured bf16 burst / 3" if bf16 else "fallback 1.9 PF / 3",
                        "note": "kernel times of concurrent streams summed"})
    ms_x = sum(d["ms_xupdate"] for d in diags)
    if ms_x > 0:
        gbs = sum(d["bytes_xupdate"] for d in diags) / (ms_x / 1e3) / 1e9
        hp = hbm or 6800.0
        kernels.append({"kernel": "k_xupdate_tc (ADMM x-update on tcgen05)", "bound": "hbm", "achieved": gbs,
                        "peak": hp, "unit": "GB/s", "frac": gbs / hp, "traffic": None,
                        "launches_per_step": sum(d["n_xupdate"] for d in diags), "ms_per_step": ms_x,
                        "peak_source": "measured HBM copy" if hbm else "fallback 6.8 TB/s",
                        "note": ("grouped replays (x-update and check launches of all problems) timed whole"
                                 if args.streams == 0 else "kernel times of concurrent streams summed")})
    kernels.sort(key=lambda k: -k["ms_per_step"])
    e2e = None
    if args.e2e_steps > 0:
        Xn = [torch.from_numpy(np.ascontiguousarray(pb.X)).pin_memory().numpy() for pb in probs]
        yn = [torch.from_numpy(np.ascontiguousarray(pb.y)).pin_memory().numpy() for pb in probs]
        t0 = time.perf_counter()
        for _ in range(args.e2e_steps):
            res = native.uoi_lasso_fit_batch(Xn, yn, streams=args.streams, **kw)
            _ = sum(float(np.asarray(r["beta"]).sum()) for r in res)
        t1 = time.perf_counter()
        e2e = {"value": args.e2e_steps * count / (t1 - t0), "unit": "fits/s",
               "h2d_bytes_per_step": int(sum(pb.X.nbytes + pb.y.nbytes for pb in probs)),
               "d2h_bytes_per_step": int(sum(pb.X.shape[1] * 8 for pb in probs))}
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        # the oracle on the median problem (by n p^2), scaled to the batch by n p^2
        work = [pb.X.shape[0] * pb.X.shape[1] ** 2 for pb in probs]
        k = int(np.argsort(work)[len(work) // 2])
        threads, listed = host_cores()
        fps, sps, desc = cpu_sample(w, np.ascontiguousarray(probs[k].X),
                                    np.ascontiguousarray(probs[k].y.reshape(-1, 1)), threads=threads)
        t_batch = sum(work) / work[k] / fps
        cpu = {"value": count / t_batch, "unit": "fits/s", "cores": threads, "host_cpus": listed,
               "kind": "oracle",
               "sample": f"problem {k} of the batch ({desc}), scaled by n p^2 to all {count}"}
    if rank == 0:
        ns = [pb.X.shape[0] for pb in probs]
        ps = [pb.X.shape[1] for pb in probs]
        line = {"metric": METRIC, "value": fits_s, "unit": "fits/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": DTYPE_MIXED if args.precision == "mixed" else "f64", "data": "synthetic",
                "config": {"workload": w.name, "problems": count, "n_range": [min(ns), max(ns)],
                           "p_range": [min(ps), max(ps)], "B1": w.B1, "q": w.q, "B2": w.B2,
                           "precision": args.precision, "warm_start": args.warm,
                           "batch_mode": "grouped" if args.streams == 0 else f"{args.streams} worker streams",
                           "parallelism": "replicas" if world > 1 else "single",
                           "l2": "inputs larger than L2 (%.0f MB of designs)" % (sum(pb.X.nbytes for pb in probs) / 1e6)},
                "solves_per_s": fits_s * w.B1 * w.q,
                "roofline": kernels[0] if kernels else None, "roofline_other": kernels[1:],
                "stage_ms": {k2: float(np.sum([d[f"ms_{k2}"] for d in diags]))
                             for k2 in ("gram", "factor", "admm", "estimation")},
                "clocks": clocks, "gpu_launches": int(sum(d["gpu_launches"] for d in diags)) * args.steps,
                "e2e": e2e, "cpu_baseline": cpu}
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
