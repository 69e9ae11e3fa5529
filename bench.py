#!/usr/bin/env python
"""Benchmark: rank-one SVD updates per second on one GB300, square n = 8192, in the
mixed form (split-BF16 tensor-core products, FP64 roots) next to the plain FP64 form
on the same GPU in the same run.

Workload: A = U diag(sigma) V^T with Haar U, V (8192 x 8192) and sigma log-uniform in
[1e-4, 1]; each step applies one rank-one update a b^T (a, b ~ N(0,1)) to the previous
result (chained updates, Alg. 6.1), inputs resident in HBM.  U and V are 512 MiB
each, larger than L2, so no flush is needed between steps.

One JSON line on stdout (rank 0).  `value` is whole-job updates/s (device-timed with
CUDA events on the library's stream); `fp64` is the plain FP64 form on the same inputs,
with its own timed region, roofline, clock record and end-to-end figure; `e2e` is the
same metric through the host-buffer entry point (copies inside the timed region);
`roofline` is for the dominant product kernel, whose launches are timed by event pairs
on their own stream inside the timed region, against App. D's algorithmic operation
count; `cpu_baseline` is the CPU oracle on a bounded, extrapolated sample of the same
update.

--impl reference times the CPU oracle (the reference arm of this comparison) instead.
Under torchrun every rank runs an independent replica (no collective in the data path).
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

MODES = {"fp64": 0, "bf16x3": 1, "fp16x2": 2}
# bf16x3: 3-term BF16 split products; fp16x2: 2-term FP16 split at a power-of-two scale per
# tile; both with FP32 accumulation and FP64 roots
DTYPES = {"fp64": "f64", "bf16x3": "bf16x3", "fp16x2": "fp16x2"}
METRIC = "rank-1 SVD updates/s at n=8192 (mixed vs FP64, same GPU) + p99 latency"


def bench_config(args, ws):
    n = args.n
    return {"workload": "square n=%d, Haar U/V, sigma log-uniform [1e-4,1], chained "
                        "N(0,1) rank-one updates" % n,
            "n": n, "mode": args.mode, "eps": args.eps,
            "l2": "inputs larger than L2 (U, V %d MiB each)" % (8 * n * n >> 20),
            "parallelism": "replicas" if ws > 1 else "single"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=8192)
    ap.add_argument("--mode", default="bf16x3", choices=list(MODES))
    ap.add_argument("--fp64-steps", type=int, default=10)
    ap.add_argument("--no-fp64", action="store_true")
    ap.add_argument("--no-alt", action="store_true",
                    help="skip the other split form's sub-line (fp16x2 beside bf16x3 and back)")
    ap.add_argument("--eps", type=float, default=1e-12)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--cpu-cols", type=int, default=64)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-lanes", type=int, default=16)
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--serve-seconds", type=float, default=10.0)
    ap.add_argument("--serve-rates", default="100,300,2000",
                    help="offered Poisson rates (updates/s) of the serving sweep")
    ap.add_argument("--serve-group", type=int, default=4)
    return ap.parse_args()


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 25 ms from before the
    warm-up until after the timed region.  Each sample carries nvidia-smi's own
    timestamp (the time of arrival where that does not parse); stop() summarises the
    samples that fall inside the host wall-clock window of the timed region."""

    Q = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    NAMES = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]

    def __init__(self, gpu: int, interval_ms: int = 10):
        self.gpu = gpu
        self.interval_ms = interval_ms
        self.proc = None
        self.lines = []  # (arrival time, line)

    def start(self, wait_s: float = 3.0):
        """Start sampling; wait (at most wait_s) for the first sample."""
        self.lines = []
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits",
                                          "-lms", str(self.interval_ms)],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        t_end = time.time() + wait_s
        while not self.lines and time.time() < t_end and self.proc.poll() is None:
            time.sleep(0.005)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    @staticmethod
    def _stamp(text, arrival):
        import datetime
        try:
            return datetime.datetime.strptime(text.strip(), "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except Exception:
            return arrival

    def stop(self, window=None):
        """Summary of the samples taken in `window` = (t0, t1), host wall-clock seconds
        (all samples when window is None).  Where none fell inside, the samples within
        250 ms of it are used and in_window is false."""
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        try:
            return self._summary(window)
        except Exception as e:  # the record is evidence, never a reason to lose the line
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock record unreadable: %s" % e]}

    def _summary(self, window):
        samples = []
        for arrival, ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 10:
                continue
            try:
                sm, smax = float(f[2]), float(f[3])
            except ValueError:
                continue
            reasons = {nm for nm, v in zip(self.NAMES, f[6:10]) if v.lower() == "active"}
            samples.append((self._stamp(f[0], arrival), sm, smax, reasons))
        chosen, in_window = samples, None
        if window is not None:
            t0, t1 = window
            chosen = [x for x in samples if t0 <= x[0] <= t1]
            in_window = bool(chosen)
            if not chosen:
                chosen = [x for x in samples if t0 - 0.25 <= x[0] <= t1 + 0.25]
        out = {"sm_mhz": float(np.median([x[1] for x in chosen])) if chosen else None,
               "sm_max_mhz": float(max(x[2] for x in chosen)) if chosen else None,
               "reasons": sorted(set().union(*[x[3] for x in chosen])) if chosen else [],
               "samples": len(chosen)}
        if window is not None:
            out["in_window"] = in_window
            out["window_ms"] = round((window[1] - window[0]) * 1e3, 3)
            out["interval_ms"] = self.interval_ms
        return out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_sample(U, S, V, a, b, ncols):
    """The oracle's update on a bounded sample: the four eigen-updates (STEPs 4-7) with
    all roots, z vectors and norms, and `ncols` sampled output columns of each product;
    the full update time is extrapolated linearly in columns.  Returns (seconds_full,
    seconds_spent, description)."""
    import oracle
    m, n = U.shape[0], V.shape[0]
    t_spent0 = time.perf_counter()
    t0 = time.perf_counter()
    p = oracle.gemv_t(U, a)
    q = oracle.gemv_t(V, b)
    t_gemv = time.perf_counter() - t0
    alpha, beta = float(a @ a), float(b @ b)
    r1, r2, Qu = oracle.schur2(beta)
    r3, r4, Qv = oracle.schur2(alpha)
    sq = S * q[:m]
    z1 = Qu[0, 0] * p + Qu[1, 0] * sq
    z2p = Qu[0, 1] * p + Qu[1, 1] * sq
    sp = np.concatenate([S * p, np.zeros(n - m)])
    z3 = Qv[0, 0] * q + Qv[1, 0] * sp
    z4p = Qv[0, 1] * q + Qv[1, 1] * sp
    Dv = np.concatenate([S ** 2, np.zeros(n - m)])
    total = t_gemv
    plan = [(U, S ** 2, z1, r1, z2p, m), (None, None, None, r2, None, m),
            (V, Dv, z3, r3, z4p, n), (None, None, None, r4, None, n)]
    carry = None
    for i, (X, d, z, rho, znext, N) in enumerate(plan):
        if X is None:  # second solve of the side: poles and z from the first
            d, z = carry
            X = np.asfortranarray(np.random.default_rng(i).standard_normal((N, N)))
        t0 = time.perf_counter()
        if znext is not None:
            lam, zrow = oracle.rank_one_update_z(znext[None, :], d, z, rho)
            carry = (lam, zrow[0])
        else:
            lam = oracle.rank_one_eig(d, z, rho, vectors=False)
        t_solve = time.perf_counter() - t0
        cols = np.linspace(0, N - 1, ncols).astype(np.int32)
        t0 = time.perf_counter()
        oracle.rank_one_update_z(X, d, z, rho, cols=cols)
        t_sample = time.perf_counter() - t0
        per_col = max(t_sample - t_solve, 0.0) / ncols
        total += t_solve + per_col * N
    spent = time.perf_counter() - t_spent0
    desc = ("oracle (bisection roots, dense product): all roots, z and norms of the 4 "
            "eigen-updates plus %d sampled output columns per product, extrapolated "
            "linearly to all columns (extrapolated)" % ncols)
    return total, spent, desc


def make_inputs(n, seed, device, steps):
    from paper_1707_08369_gb300 import workloads as wl
    U, S, V, a0, b0 = wl.loguniform_sq(n, seed=seed, device=device)
    g = wl.rng(seed + 7)
    ab = [(g.standard_normal(n), g.standard_normal(n)) for _ in range(steps)]
    return U, S, V, ab


def run_reference(args, ws, rank):
    if rank != 0:
        return
    import oracle
    oracle.build()
    n = args.n
    U, S, V, ab = make_inputs(n, 170708369 + 2, None, 1)
    a, b = ab[0]
    ncols = 16
    times = []
    for i in range(args.warmup + args.steps):
        full, spent, desc = oracle_sample(U, S, V, a, b, ncols)
        if i >= args.warmup:
            times.append(full)
    t = float(np.mean(times))
    value = 1.0 / t
    line = {"impl": "reference", "metric": METRIC, "value": value,
            "unit": "updates/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": bench_config(args, ws),
            "cpu_baseline": {"value": value, "unit": "updates/s", "cores": oracle.num_threads(),
                             "kind": "oracle", "sample": desc.replace("%d" % ncols, str(ncols))},
            "e2e": {"value": value, "unit": "updates/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def load_peaks():
    """Measured peaks of this machine's GB300 (written next to the repository by the
    driver); the documented fallback figures when the file is absent."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return pk, "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def recorded_traffic(n, mode_name):
    """DRAM bytes per launch of the output-stage kernel from the committed ncu summary
    (profiles/umma_out_traffic.json), if it was taken on this workload and the kernel
    source is unchanged since (SHA-256 of csrc/svdup_mixed.cu); else None."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", "umma_out_traffic.json")) as f:
            rec = json.load(f)
        with open(os.path.join(ROOT, "paper_1707_08369_gb300", "csrc", "svdup_mixed.cu"), "rb") as f:
            sha = hashlib.sha256(f.read()).hexdigest()
    except Exception:
        return None
    if rec.get("source_sha256") != sha or rec.get("n") != n or rec.get("mode") != mode_name:
        return None
    return rec.get("bytes_per_launch")


def fp64_peak_tflops(sm_mhz):
    """FP64 (DFMA) peak from unit counts and clock: 152 SMs x 2 DFMA per SM per clock
    x 2 flops (1.26 TFLOP/s at 2070 MHz)."""
    return 152 * 2 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


STAGE_KERNELS = {"p2m": "P2M", "m2l": "M2L", "out": "OUT"}


def roofline_of(kernels, mode, clk, peaks, peak_src, n, mode_name):
    """Roofline of the dominant product kernel, from its own event timers over the timed
    region: achieved = the algorithmic flops of its launches (App. D's operation count,
    14 N p multiply-adds per right-hand side for the whole FMM, of which STEPs 9-10 fall
    to the output stage) / their summed duration.  The executed flops (the six split BF16
    partial products, padding included) and the useful flops of the flat partition are
    reported beside it."""
    dom = max(kernels, key=lambda k: kernels[k][0])
    ms, cnt, useful, executed, alg = kernels[dom]
    cnt = max(int(cnt), 1)
    per_launch_s = ms / cnt / 1e3
    per = lambda fl: fl / cnt / per_launch_s / 1e12
    if mode == 0:
        peak = fp64_peak_tflops(clk.get("sm_mhz") if clk else None)
        # (FP64: the translation stage is the hierarchy's shifts and translations)
        kname = "k_tree_gemm<UP/M2L/DOWN>" if dom == "m2l" else "k_gemm_f64<%s>" % STAGE_KERNELS[dom]
        r = {"kernel": kname, "bound": "alu",
             "achieved": per(alg), "peak": peak, "unit": "TFLOP/s", "frac": per(alg) / peak,
             "traffic": None, "useful_tflops": per(useful), "useful_frac": per(useful) / peak,
             "peak_source": "FP64 pipe from unit counts and the sampled SM clock "
                            "(152 SMs x 2 DFMA/clk x 2 flops), not a measured figure"}
    else:
        peak = float(peaks["bf16_tflops_sustained"])
        r = {"kernel": "k_umma<%s>" % STAGE_KERNELS[dom], "bound": "tensor",
             "achieved": per(alg), "peak": peak, "unit": "TFLOP/s", "frac": per(alg) / peak,
             "traffic": recorded_traffic(n, mode_name) if dom == "out" else None,
             "executed_tflops": per(executed), "executed_frac": per(executed) / peak,
             "useful_tflops": per(useful),
             "peak_source": "bf16_tflops_sustained, %s (kernel timed inside a long step)" % (
                 "of MEASURED_PEAKS.json" if peak_src == "measured" else
                 "fallback figure (MEASURED_PEAKS.json absent)")}
    r.update({"launches": cnt, "ms_per_launch": ms / cnt,
              "alg_flops_per_launch": alg / cnt,
              "work": "algorithmic flops: App. D's 14 N p multiply-adds per row for N points at "
                      "order p, split 2:5:7 over P2M, M2L, OUT; N = the product's non-deflated "
                      "size, 2 flops per multiply-add; launch durations from event pairs on the "
                      "kernel's own stream inside the timed region"})
    return r


def timed_updates(sv, h, stream, tU, tS, tV, ta, tb, mode, eps, warmup, steps, ws, dev, clocks=None,
                  stage_steps=1):
    """W untimed then K timed chained updates on the handle's stream; returns per-update
    latencies (ms), the total (ms), the launch count, the stage timers and how many
    updates they cover, the clock record, and the product kernels' own timers over the
    timed region.  The timed updates run as in use (the left- and right-hand problems on
    their streams), with the kernel timers on: an event pair around each product-stage
    kernel on the stream it runs on, which leaves the schedule as it is.  The per-stage
    breakdown needs one stream, so it comes from `stage_steps` further updates after the
    timed region."""
    import torch
    with torch.cuda.stream(stream):
        if clocks is not None:
            clocks.start()  # running, with a first sample, before the warm-up
        for i in range(warmup):
            h.update(tU, tS, tV, ta[i], tb[i], eps=eps, mode=mode, check=False)
        rc = h.sync()
        if rc != 0:
            raise SystemExit("warm-up update failed: %s" % sv.error_string(rc))
        h.timing(sv.TIMING_KERNELS)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
        launches0 = h.launch_count()
        if ws > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)
        t_wall0 = time.time()
        ev[0].record(stream)
        for i in range(steps):
            j = warmup + i
            h.update(tU, tS, tV, ta[j], tb[j], eps=eps, mode=mode, check=False)
            ev[i + 1].record(stream)
        torch.cuda.synchronize(dev)
        t_wall1 = time.time()
        if ws > 1:
            torch.distributed.barrier()
        clk = clocks.stop((t_wall0, t_wall1)) if clocks is not None else None
        launches = h.launch_count() - launches0
        rc = h.sync()
        if rc != 0:
            raise SystemExit("timed update failed: %s" % sv.error_string(rc))
        kernels = h.timing_read()
        alg = h.timing_read_alg()
        kernels = {k: v + (alg[k],) for k, v in kernels.items() if k in ("p2m", "m2l", "out")}
        h.timing(False)
        stages = None
        if stage_steps > 0:
            h.timing(True)
            for i in range(stage_steps):
                j = (warmup + steps + i) % len(ta)
                h.update(tU, tS, tV, ta[j], tb[j], eps=eps, mode=mode, check=False)
            rc = h.sync()
            if rc != 0:
                raise SystemExit("timing update failed: %s" % sv.error_string(rc))
            stages = h.timing_read()
            h.timing(False)
    lat = np.array([ev[i].elapsed_time(ev[i + 1]) for i in range(steps)])
    total_ms = float(ev[0].elapsed_time(ev[-1]))
    if ws > 1:
        total_ms = max_over_ranks(total_ms, dev)
    return lat, total_ms, launches, (stages, stage_steps), clk, kernels


def max_over_ranks(ms, device):
    """The slowest rank's time (every rank runs an independent replica; the whole-job
    rate is the units of all ranks over this time).  Works on any process-group backend
    (NCCL on the GPU, gloo on the CPU)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_rate(units_per_rank, ms, ws):
    """Whole-job units per second: every rank did units_per_rank units in at most ms."""
    return ws * units_per_rank / (ms / 1e3)


def accuracy_report(sv, h, stream, upload, ta, tb, eps, modes, dev):
    """One update from the same inputs in the FP64 form and in each mode of `modes`;
    each mixed form's errors against the FP64 form, and invariants of each output
    measured with random probes x (n x 4, FP64 on the device): ||U^T U x - x||,
    ||V^T V x - x|| and the reconstruction ||Ahat Vhat x - Uhat Shat x|| / (sigma_max ||x||)
    with Ahat = U S V^T + a b^T applied factor by factor."""
    import torch
    outs = {}
    names = {v: k for k, v in MODES.items()}
    with torch.cuda.stream(stream):
        U0, S0, V0 = upload()
        for m in sorted({0, *modes}):
            tU, tS, tV = upload()
            h.update(tU, tS, tV, ta[0], tb[0], eps=eps, mode=m, check=True)
            outs[m] = (tU, tS, tV)
        torch.cuda.synchronize(dev)
        gen = torch.Generator(device=dev)
        gen.manual_seed(170708369)
        n, m_ = V0.shape[0], U0.shape[0]
        x = torch.randn(m_, 4, dtype=torch.float64, device=dev, generator=gen)
        y = torch.randn(n, 4, dtype=torch.float64, device=dev, generator=gen)
        rep = {}
        for mm, (Un, Sn, Vn) in outs.items():
            Vm = Vn[:, :m_]
            ortU = float(torch.linalg.norm(Un.t() @ (Un @ x) - x) / torch.linalg.norm(x))
            ortV = float(torch.linalg.norm(Vn.t() @ (Vn @ y) - y) / torch.linalg.norm(y))
            w = Vm @ x
            lhs = U0 @ (S0[:, None] * (V0[:, :m_].t() @ w)) + ta[0][:, None] * (tb[0][None, :] @ w)
            rec = float(torch.linalg.norm(lhs - Un @ (Sn[:, None] * x)) / (Sn[0] * torch.linalg.norm(x)))
            rep[mm] = {"orth_U": ortU, "orth_V": ortV, "recon": rec}
        res = {"probe": "4 Gaussian probe vectors; norms are 2-norms of the probe block",
               "fp64": rep[0]}
        U64, S64, V64 = outs[0]
        for mm in modes:
            if mm == 0:
                continue
            Um, Sm, Vm2 = outs[mm]
            res[names[mm]] = dict(rep[mm], vs_fp64={
                "sigma_max_rel": float((Sm - S64).abs().max() / S64[0]),
                "U_max_abs": float((Um - U64).abs().max()),
                "V_max_abs": float((Vm2[:, :m_] - V64[:, :m_]).abs().max())})
    del outs
    return res


def refine_report(sv, h, stream, upload, ta, tb, eps, mode, dev):
    """The precision form's refinement step (one Newton-Schulz step on Uhat and on Vhat,
    forced with tolerance 0): its cost (an update with the step minus one without, each
    timed by CUDA events after a warm-up call) and the probe invariants after it."""
    import torch
    h.set_refine_tol(0.0)
    ms = {}
    with torch.cuda.stream(stream):
        for flags in (sv.REFINE, 0, sv.REFINE):  # the first call grows the workspace
            tU, tS, tV = upload()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            h.update(tU, tS, tV, ta[0], tb[0], eps=eps, mode=mode | flags, check=True)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms[flags] = e0.elapsed_time(e1)
        before = h.refine_residuals()
        gen = torch.Generator(device=dev)
        gen.manual_seed(170708369)
        x = torch.randn(tU.shape[1], 4, dtype=torch.float64, device=dev, generator=gen)
        y = torch.randn(tV.shape[1], 4, dtype=torch.float64, device=dev, generator=gen)
        oU = float(torch.linalg.norm(tU.t() @ (tU @ x) - x) / torch.linalg.norm(x))
        oV = float(torch.linalg.norm(tV.t() @ (tV @ y) - y) / torch.linalg.norm(y))
    h.set_refine_tol(1e-6)
    return {"step_ms": ms[sv.REFINE] - ms[0], "update_ms_with_step": ms[sv.REFINE],
            "probe_residual_before": {"U": before[0], "V": before[1]},
            "after": {"orth_U": oU, "orth_V": oV},
            "note": "one Newton-Schulz step X (3I - X^T X)/2 on Uhat and Vhat, forced "
                    "(tolerance 0); E in 3-term BF16 split, X E in one BF16 product"}


def batched_form(sv, dev, mode, eps, count, steps, warmup, lanes):
    """The batching form: `count` independent square updates, n log-uniform in
    [32, 1024], each A Gaussian (its SVD taken on the device with torch.linalg.svd,
    input preparation only), a, b Gaussian.  The product path is autotuned first; the
    batch is recorded once into a CUDA graph and launched steps times (chained updates
    of all problems per launch); the same batch without a graph is timed once."""
    import torch
    from paper_1707_08369_gb300 import workloads as wl
    ns = wl.uneven_sizes(count, 32, 1024, seed=wl.BASE_SEED + 3)
    g = torch.Generator(device=dev)
    g.manual_seed(wl.BASE_SEED + 3)
    items = []
    for n in ns:
        n = int(n)
        A = torch.randn(n, n, dtype=torch.float64, device=dev, generator=g)
        U, S, Vh = torch.linalg.svd(A)
        a = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
        b = torch.randn(n, dtype=torch.float64, device=dev, generator=g)
        # column-major U and V = Vh^T (a transposed row-major tensor is column-major)
        items.append((U.t().contiguous().t(), S.contiguous(), Vh.contiguous().t(), a, b))
    torch.cuda.synchronize(dev)
    h = sv.Handle(dev.index)
    t0 = time.perf_counter()
    tuned = h.autotune(mode, nmax=1024)
    tile128 = h.tile_tuning(mode)
    t_tune = time.perf_counter() - t0
    t0 = time.perf_counter()
    bt = h.batch_plan(items, eps=eps, mode=mode, lanes=lanes)
    t_plan = time.perf_counter() - t0
    for _ in range(warmup):
        bt.launch(check=False)
    rc = h.sync()
    if rc:
        raise SystemExit("batched warm-up failed: %s" % sv.error_string(rc))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize(dev)
    e0.record(h.stream)
    for _ in range(steps):
        bt.launch(check=False)
    e1.record(h.stream)
    torch.cuda.synchronize(dev)
    rc = h.sync()
    if rc:
        raise SystemExit("batched run failed: %s" % sv.error_string(rc))
    ms = e0.elapsed_time(e1) / steps
    kernels = bt.kernels()
    bt.close()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    h.update_batched(items, eps=eps, mode=mode, lanes=lanes)
    t_nograph = time.perf_counter() - t0
    h.close()
    return {"workload": "%d independent square updates, n log-uniform in [32, 1024], Gaussian A "
                        "(SVD by torch.linalg.svd on the device as input), N(0,1) a, b" % count,
            "value": count / (ms / 1e3), "unit": "updates/s", "ms_per_batch": ms, "steps": steps,
            "lanes": lanes, "graph_kernels": kernels, "plan_s": t_plan,
            "autotune": {"dense_max": tuned[0], "leaf128_min": tuned[1],
                         "dense_tile128_min": tile128, "seconds": t_tune},
            "no_graph_ms_per_batch": t_nograph * 1e3}


def serving_form(sv, dev, mode, eps, seconds, rates, nmats, lanes, group, seed):
    """The serving form: `nmats` resident SVDs of m x 2m matrices, m log-uniform in
    [1024, 4096], spectrum log-uniform in [1e-4, 1] with Haar U, V (QR of Gaussians on the
    device, input preparation only); rank-one updates with N(0,1) a, b arrive as a
    Poisson stream for `seconds` at each offered rate, each for a uniformly chosen
    matrix, and are submitted to the serving engine as they arrive (lanes take up to
    `group` requests of one size class per cycle).  The vectors come from a pool of 32
    seeded N(0,1) pairs per matrix.  Per rate: the sustained updates/s (completed / time
    from the first arrival to the last completion) and the latency percentiles
    (submission to the posted result, queueing included)."""
    import torch
    g = np.random.default_rng(seed)
    ms = np.rint(1024 * 4.0 ** g.uniform(0, 1, nmats)).astype(int)
    tg = torch.Generator(device=dev)
    tg.manual_seed(seed)
    srv = sv.Server(dev.index, lanes=lanes, eps=eps, mode=mode)
    srv.set_group(group)
    live, shapes = [], []
    for m in ms:
        m = int(m)
        n = 2 * m
        U, _ = torch.linalg.qr(torch.randn(m, m, dtype=torch.float64, device=dev, generator=tg))
        V, _ = torch.linalg.qr(torch.randn(n, n, dtype=torch.float64, device=dev, generator=tg))
        S = torch.from_numpy(np.sort(10.0 ** (-4.0 * g.uniform(0, 1, m)))[::-1].copy()).to(dev)
        U, V = U.t().contiguous().t(), V.t().contiguous().t()
        live.append((U, S, V))
        shapes.append((m, n))
    torch.cuda.synchronize(dev)
    ids = [srv.register(U, S, V) for U, S, V in live]
    pool = [[(g.standard_normal(m), g.standard_normal(n)) for _ in range(32)] for m, n in shapes]
    # warm the lanes' workspaces with one update per matrix (not timed)
    for i in range(nmats):
        srv.wait(srv.submit(ids[i], *pool[i][0]))
    out = []
    for rate in rates:
        nreq = max(1, int(rate * seconds))
        gaps = g.exponential(1.0 / rate, nreq)
        which = g.integers(0, nmats, nreq)
        pick = g.integers(0, 32, nreq)
        g0 = srv.group_stats()
        t0 = time.perf_counter()
        arrive = t0 + np.cumsum(gaps)
        tickets = []
        for k in range(nreq):
            while time.perf_counter() < arrive[k]:
                pass
            i = int(which[k])
            tickets.append(srv.submit(ids[i], *pool[i][int(pick[k])]))
        lats = []
        for t in tickets:
            st, lat = srv.wait(t)
            if st:
                raise SystemExit("serving update failed: %s" % sv.error_string(st))
            lats.append(lat)
        t_end = time.perf_counter()
        g1 = srv.group_stats()
        lats = np.array(lats)
        cyc = g1["groups"] - g0["groups"]
        out.append({"offered_per_s": rate, "requests": nreq, "seconds": seconds,
                    "value": nreq / (t_end - t0), "unit": "updates/s (sustained)",
                    "latency_ms": {"p50": float(np.percentile(lats, 50)),
                                   "p99": float(np.percentile(lats, 99))},
                    "mean_group": (g1["grouped"] - g0["grouped"]) / max(cyc, 1)})
    stats = srv.stats()
    srv.close()
    return {"workload": "%d resident SVDs m x 2m, m log-uniform in [1024, 4096], sigma "
                        "log-uniform [1e-4, 1]; Poisson arrivals of N(0,1) rank-one updates "
                        "(pool of 32 pairs per matrix)" % nmats,
            "lanes": lanes, "group_max": group, "sweep": out,
            "max_in_flight": stats["max_in_flight"], "max_workspace_bytes": stats["max_ws_bytes"]}


def main():
    args = parse()
    ws, rank, local = dist_env()
    if args.impl == "reference":
        run_reference(args, ws, rank)
        return
    import torch
    import paper_1707_08369_gb300 as sv
    from paper_1707_08369_gb300 import build as svbuild
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    svbuild.build()
    sv.load()
    n = args.n
    mode = MODES[args.mode]
    dev = torch.device("cuda", local)
    steps_total = args.warmup + args.steps
    U, S, V, ab = make_inputs(n, 170708369 + 2 + 1000 * rank, dev, steps_total)
    U_h, S_h, V_h = (U, S, V) if (rank == 0 and not args.no_cpu) else (None, None, None)

    def upload():
        tU = torch.from_numpy(np.asfortranarray(U).T.copy()).to(dev).t()
        tV = torch.from_numpy(np.asfortranarray(V).T.copy()).to(dev).t()
        tS = torch.from_numpy(S.copy()).to(dev)
        return tU, tS, tV

    ta = [torch.from_numpy(a).to(dev) for a, _ in ab]
    tb = [torch.from_numpy(b).to(dev) for _, b in ab]
    stream = torch.cuda.Stream(device=dev)
    h = sv.Handle(local, stream=stream)
    tU, tS, tV = upload()
    clocks = ClockSampler(local)
    lat, total_ms, launches, (stages, stage_n), clk, kern = timed_updates(
        sv, h, stream, tU, tS, tV, ta, tb, mode, args.eps, args.warmup, args.steps, ws, dev, clocks)
    value = replica_rate(args.steps, total_ms, ws)
    peaks, peak_src = load_peaks()
    roofline = roofline_of(kern, mode, clk, peaks, peak_src, n, args.mode)
    stage_ms = {k: round(v[0] / stage_n, 3) for k, v in stages.items()}

    def e2e_form(m_, steps_):
        """The same metric end to end through the host-buffer entry point: every step
        copies U, S, V, a, b from pinned host memory to the device and the results back
        (host wall clock around the call, which waits for completion)."""
        pU = torch.empty((n, n), dtype=torch.float64, pin_memory=True).numpy()
        pV = torch.empty((n, n), dtype=torch.float64, pin_memory=True).numpy()
        pS = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        pa = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        pb = torch.empty(n, dtype=torch.float64, pin_memory=True).numpy()
        pUf = pU.T  # column-major views of the pinned buffers
        pVf = pV.T
        pUf[...] = tU.cpu().numpy()
        pVf[...] = tV.cpu().numpy()
        pS[...] = tS.cpu().numpy()
        times = []
        for i in range(steps_ + 1):  # the first call is an untimed warm-up
            pa[...] = ab[i % len(ab)][0]
            pb[...] = ab[i % len(ab)][1]
            t0 = time.perf_counter()
            h.update_host(pUf, pS, pVf, pa, pb, eps=args.eps, mode=m_)
            if i > 0:
                times.append(time.perf_counter() - t0)
        t = float(np.mean(times))
        if ws > 1:
            t = max_over_ranks(t, dev)
        return {"value": ws / t, "unit": "updates/s", "steps": steps_,
                "h2d_bytes_per_step": 8 * (2 * n * n + 3 * n),
                "d2h_bytes_per_step": 8 * (2 * n * n + n)}

    # the plain FP64 form on the same GPU, same workload (the comparison the metric names):
    # its own timed region, clock record, roofline and end-to-end figure
    fp64 = None
    if mode != 0 and not args.no_fp64:
        del tU, tV
        tU, tS, tV = upload()
        w64 = min(args.warmup, 3)
        k64 = min(max(3, args.fp64_steps), steps_total - w64)
        clocks64 = ClockSampler(local, interval_ms=25)
        lat64, tot64, _, _, clk64, kern64 = timed_updates(
            sv, h, stream, tU, tS, tV, ta, tb, 0, args.eps, w64, k64, ws, dev, clocks64,
            stage_steps=0)
        k64 = len(lat64)
        v64 = ws * k64 / (tot64 / 1e3)
        fp64 = {"value": v64, "unit": "updates/s", "steps": k64, "warmup": w64,
                "ms_per_step": tot64 / k64,
                "latency_ms": {"p50": float(np.percentile(lat64, 50)),
                               "p99": float(np.percentile(lat64, 99))},
                "mixed_over_fp64": value / v64,
                "roofline": roofline_of(kern64, 0, clk64, peaks, peak_src, n, "fp64"),
                "clocks": clk64}
        if not args.no_e2e and args.e2e_steps > 0:
            fp64["e2e"] = e2e_form(0, args.e2e_steps)
        del tU, tV
        tU, tS, tV = upload()

    # the other split form on the same GPU and workload: its own timed region
    alt = None
    alt_name = {"bf16x3": "fp16x2", "fp16x2": "bf16x3"}.get(args.mode)
    if alt_name and not args.no_alt:
        del tU, tV
        tU, tS, tV = upload()
        w2 = min(args.warmup, 3)
        k2 = min(args.steps, steps_total - w2)
        lat2, tot2, _, _, clk2, kern2 = timed_updates(
            sv, h, stream, tU, tS, tV, ta, tb, MODES[alt_name], args.eps, w2, k2, ws, dev,
            ClockSampler(local), stage_steps=0)
        v2 = ws * len(lat2) / (tot2 / 1e3)
        alt = {"mode": alt_name, "value": v2, "unit": "updates/s", "steps": len(lat2),
               "warmup": w2, "ms_per_step": tot2 / len(lat2),
               "latency_ms": {"p50": float(np.percentile(lat2, 50)),
                              "p99": float(np.percentile(lat2, 99))},
               "roofline": roofline_of(kern2, MODES[alt_name], clk2, peaks, peak_src, n, alt_name),
               "clocks": clk2}
        if fp64:
            alt["over_fp64"] = v2 / fp64["value"]
        del tU, tV
        tU, tS, tV = upload()

    acc_modes = [mode] + ([MODES[alt_name]] if alt else [])
    accuracy = None if args.no_accuracy else accuracy_report(
        sv, h, stream, upload, ta, tb, args.eps, acc_modes, dev)
    refine = None
    if mode != 0 and not args.no_accuracy:
        refine = {args.mode: refine_report(sv, h, stream, upload, ta, tb, args.eps, mode, dev)}
        if alt:
            refine[alt_name] = refine_report(sv, h, stream, upload, ta, tb, args.eps,
                                             MODES[alt_name], dev)
    batched = None
    if not args.no_batched and ws == 1:
        batched = batched_form(sv, dev, mode, args.eps, args.batch_count, 5, 2, args.batch_lanes)
    serving = None
    if not args.no_serving and ws == 1:
        serving = serving_form(sv, dev, mode, args.eps, args.serve_seconds,
                               [float(r) for r in args.serve_rates.split(",")], 16, 8,
                               args.serve_group, 170708369 + 4)

    # end-to-end through the host-buffer entry point (pinned host memory)
    e2e = None
    if not args.no_e2e and args.e2e_steps > 0:
        e2e = e2e_form(mode, args.e2e_steps)

    cpu = None
    if rank == 0 and not args.no_cpu:
        import oracle
        oracle.build()
        full, spent, desc = oracle_sample(U_h, S_h, V_h, ab[0][0], ab[0][1], args.cpu_cols)
        cpu = {"value": 1.0 / full, "unit": "updates/s", "cores": oracle.num_threads(), "kind": "oracle",
               "sample": desc + "; %.1f s of CPU time spent" % spent}

    if rank == 0:
        line = {"metric": METRIC,
                "value": value, "unit": "updates/s",
                "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": DTYPES[args.mode], "data": "synthetic",
                "config": bench_config(args, ws),
                "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
                "fp64": fp64,
                (alt_name or "alt"): alt,
                "accuracy": accuracy,
                "refine": refine,
                "batched": batched,
                "serving": serving,
                "stage_ms_per_update": stage_ms,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": int(launches), "clocks": clk}
        print(json.dumps(line), flush=True)
    h.close()
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
