"""Benchmark: OT solves/s of PINS on one GB300 (Algorithm 2, whole solve per step).

Workload (default): a single dense instance, m = n = 4096, points from an
8-component 2-D Gaussian mixture (means U[0,1]^2, sigma 0.05), squared-Euclidean
cost normalised to max 1, a, b ~ Dirichlet(1), eta = 1e-2, the paper's
hyperparameters (T1 = 100, T2 = 50, K = 250, Theorem 2 sparsity budget).  One
step = one complete solve, the cost matrix already resident in HBM.  `e2e` times
the same solve through the public C ABI from pinned host buffers (cost matrix
and marginals uploaded, potentials read back) every step.

Prints one JSON line (see the repository's benchmark contract).  `--impl
reference` times the FP64 CPU oracle instead on a bounded sample.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--eta", type=float, default=1e-2)
    ap.add_argument("--K", type=int, default=250)
    ap.add_argument("--gamma", type=float, default=1.0)
    ap.add_argument("--fp64-steps", type=int, default=1,
                    help="plain FP64 solves timed for the comparison key (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--lse-roofline", type=int, default=0, metavar="N",
                    help="instead of the contract line: HBM roofline of the mixed Sinkhorn "
                         "row and column passes on an N x N dense FP32 GMM cost (N = 16384 "
                         "puts C at 1 GiB, well beyond L2)")
    ap.add_argument("--batch", type=int, default=0, metavar="P",
                    help="instead of the contract line: P stroke-histogram pairs (grids 16^2 to "
                         "64^2) through pins_solve_batch, mixed, vs plain FP64 one at a time")
    ap.add_argument("--batch-inflight", type=int, default=8)
    ap.add_argument("--fp64-seconds", type=float, default=120.0,
                    help="time budget of the FP64 one-at-a-time arm of --batch")
    ap.add_argument("--serving", action="store_true",
                    help="instead of the contract line: a served request stream (Poisson "
                         "arrivals of point-cloud pairs) with p50/p99 latency, mixed served vs "
                         "plain FP64 one at a time")
    ap.add_argument("--serve-requests", type=int, default=24)
    ap.add_argument("--serve-rate", type=float, default=100.0, help="arrivals per second")
    ap.add_argument("--serve-nmin", type=int, default=256)
    ap.add_argument("--serve-nmax", type=int, default=2048)
    ap.add_argument("--serve-inflight", type=int, default=4)
    ap.add_argument("--serve-fp64", type=int, default=-1,
                    help="requests of the stream solved by the FP64 arm (-1: all)")
    return ap.parse_args()


def whole_job_rate(t_local: float, steps: int, world: int, device: str = "cpu"):
    """Max over ranks of the timed-region length, and the whole-job rate (every
    rank ran `steps` independent solves).  Needs an initialised process group when
    world > 1 (NCCL with device='cuda' in the benchmark, gloo with 'cpu' in tests)."""
    t = float(t_local)
    if world > 1:
        import torch
        import torch.distributed as dist
        tt = torch.tensor([t], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t = float(tt.item())
    return steps * world / t, t


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while the timed region runs."""

    def __init__(self, index: int = 0):
        self.index = index
        self.samples = []
        self._stop = threading.Event()
        self._t = None

    def _run(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        while not self._stop.is_set():
            try:
                out = subprocess.run(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                      "--format=csv,noheader,nounits"], capture_output=True,
                                     text=True, timeout=5).stdout.strip()
                if out:
                    self.samples.append([x.strip() for x in out.split(",")])
            except Exception:
                pass
            self._stop.wait(0.2)

    def __enter__(self):
        self._t = threading.Thread(target=self._run, daemon=True)
        self._t.start()
        return self

    def __exit__(self, *a):
        self._stop.set()
        self._t.join(timeout=10)

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = sorted(float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit())
        mx = max(float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit())
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4)
                          if len(s) > 3 + k and s[3 + k].lower().startswith("active")})
        return {"sm_mhz": sm[len(sm) // 2] if sm else None, "sm_max_mhz": mx,
                "reasons": reasons, "samples": len(self.samples)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# kernel classes that stream the m x n matrix once per launch
MN_CLASSES = ("row_lse", "col_lse", "marginals", "trial", "key_hist", "key_compact",
              "csr_write", "certificate")
FP64_NOMINAL_TFLOPS = 1.25   # GB300 nominal FP64 rate (the measured peaks file has no FP64 figure)
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12   # FP32 units x clock, FMA = 2 flops
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of
# each class's kernel on this workload (mid-solve, caches flushed by ncu); the
# summaries with their commands are in profiles/.  Set a class to None when its
# kernel changes until it is captured again.
NCU_TRAFFIC_BYTES = {
    "cg": None,              # k_pcg_dd changed after its capture (428 288 B then)
    "trial": 67849472,       # k_marg_mx<mixed,1>  (profiles/k_marg_mx_trial_gmm4096.md)
    "row_lse": None,         # k_row_lse_mx changed after its capture (67 766 016 B then)
    "col_lse": None,         # k_col_lse_mx changed after its capture
    "key_compact": 67311360, # k_fast_collect      (profiles/sparsify_one_pass_gmm4096.md)
}


def roofline(prof, m, n, elem_bytes, cg_iters, nnz, peaks, mixed):
    """Roofline object for the class with the largest device time.

    m x n passes: algorithmic bytes = m * n * elem_bytes (the cost matrix read once;
    potentials and partials are O(m + n)); bound 'hbm' against the measured copy
    bandwidth.  CG per iteration: FP64 path 4 nnz + 14 (m + n) FP64 flops
    (off-diagonal SpMV on the CSR and CSC copies, diagonal, three dot products and
    four vector updates) against the nominal FP64 rate; mixed path (pipelined
    ordering, double-float vectors) counted as the FP32 operations the pipelined
    kernel issues (FMA = 2): 15 per stored entry of the CSR and CSC copies (a
    double-float product and compensated sum), 152 per unknown (eight
    double-float axpy updates of 15, the diagonal product and sum, the Jacobi
    scaling, three FP32 dot terms), i.e. 30 nnz + 152 (m + n), against the FP32
    peak from the unit counts and clock (152 SMs x 128 lanes x 2 x 2.07 GHz)."""
    dom, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    if cnt == 0:
        return None, dom
    t = ms / cnt / 1e3
    if dom == "cg":
        iters = cg_iters / max(cnt, 1)
        if mixed:
            per_launch = (30.0 * nnz + 152.0 * (m + n)) * iters
            peak, src = FP32_PEAK_TFLOPS, "FP32 units x clock (152 x 128 x 2 x 2.07 GHz)"
        else:
            per_launch = (4.0 * nnz + 14.0 * (m + n)) * iters
            peak, src = FP64_NOMINAL_TFLOPS, "nominal FP64 (recipe table)"
        achieved = per_launch / t / 1e12
        return {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak,
                "unit": "TFLOP/s", "frac": achieved / peak, "traffic": None,
                "peak_source": src, "avg_launch_us": t * 1e6, "launches": cnt,
                "iters_per_launch": iters,
                "note": "latency-bound: one cluster barrier and one L2 exchange per CG iteration"}, dom
    per_launch = float(m) * n * elem_bytes
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = per_launch / t / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": None,
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "avg_launch_us": t * 1e6, "launches": cnt}, dom


def workload(args):
    from paper_2502_03749_gb300 import workloads as wl
    return wl.gmm_instance(0, m=args.n, n=args.n, eta=args.eta)


def config_dict(args, w):
    return {"workload": f"dense GMM instance m=n={args.n}, squared-Euclidean cost /max, "
                        f"Dirichlet(1) marginals, eta={args.eta}",
            "m": args.n, "n": args.n, "eta": args.eta, "K": args.K, "T1": 100, "T2": 50,
            "sparsify_gamma": args.gamma, "precision": args.prec,
            "l2_note": "C is 64 MiB FP32 (mixed) / 128 MiB FP64; L2 flushed (256 MiB write) "
                       "between timed steps; one step is a whole solve (~1e4 passes over C)",
            "parallelism": "replicas" if args.gpus > 1 else "single GPU"}


# --------------------------------------------------------------------------- #
# reference arm: the FP64 CPU oracle, bounded sample
# --------------------------------------------------------------------------- #
def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    from oracle import pins_oracle as po
    w = workload(args)
    C, a, b = w.dense_cost(), w.a, w.b
    cores = 1
    # one Sinkhorn iteration (two m x n passes) of the oracle, timed until the
    # budget is spent; a solve has K*T1 of them plus the Newton passes
    t0 = time.perf_counter()
    it = 0
    F, G = np.zeros(args.n), np.zeros(args.n)
    per_step = max(1, int(args.cpu_seconds / max(args.steps + args.warmup, 1) / 0.4))
    times = []
    for step in range(args.warmup + args.steps):
        ts = time.perf_counter()
        for _ in range(per_step):
            F, _ = po.sinkhorn_row_step(C, a, F, G, args.eta, 1.0)
            G = po.sinkhorn_col_step(C, b, F, G, args.eta, 1.0)
            it += 1
        if step >= args.warmup:
            times.append((time.perf_counter() - ts) / per_step)
    t_iter = float(np.median(times))
    # a paper-default solve runs K outer iterations of T1 Sinkhorn iterations and up to
    # T2 Newton steps; each Newton step costs at least one trial pass (2 transcendentals
    # per entry) plus the gradient/sparsify passes: counted as 2 Sinkhorn iterations.
    est = args.K * (100 + 2 * 50) * t_iter
    val = 1.0 / est
    line = {"impl": "reference", "metric": "OT solves/s", "value": val, "unit": "solves/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": est * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_dict(args, w),
            "cpu_baseline": {"value": val, "unit": "solves/s", "cores": cores, "kind": "oracle",
                             "sample": f"{per_step} oracle Sinkhorn iterations per step "
                                       f"({t_iter*1e3:.1f} ms each, m=n={args.n}); a solve "
                                       f"counted as K*(T1 + 2*T2) = {args.K*200} iterations"},
            "e2e": {"value": val, "unit": "solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# our arm
# --------------------------------------------------------------------------- #
def cpu_baseline_sample(args, w):
    """The oracle timed on a bounded sample of the same workload (rank 0, N = 1)."""
    from oracle import pins_oracle as po
    C, a, b = w.dense_cost(), w.a, w.b
    F, G = np.zeros(args.n), np.zeros(args.n)
    iters, t0 = 0, time.perf_counter()
    while iters == 0 or time.perf_counter() - t0 < args.cpu_seconds:
        F, _ = po.sinkhorn_row_step(C, a, F, G, args.eta, 1.0)
        G = po.sinkhorn_col_step(C, b, F, G, args.eta, 1.0)
        iters += 1
    t_iter = (time.perf_counter() - t0) / iters
    est = args.K * (100 + 2 * 50) * t_iter
    return {"value": 1.0 / est, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{iters} oracle Sinkhorn iterations on the m=n={args.n} instance "
                      f"({t_iter*1e3:.1f} ms each); a solve counted as K*(T1 + 2*T2) = "
                      f"{args.K*200} such iterations"}


def run_ours(args):
    import torch
    from paper_2502_03749_gb300 import pins
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    w = workload(args)
    C32 = w.dense_cost().astype(np.float32) if args.prec == "mixed" else w.dense_cost()
    # inputs resident on the device
    Cd = torch.from_numpy(C32).cuda()
    ad = torch.from_numpy(w.a).cuda()
    bd = torch.from_numpy(w.b).cuda()
    pdev = pins.make_problem("dense", ad, bd, C=Cd, on_device=True)
    stream = torch.cuda.Stream()
    # timed solves run without per-launch events (recording them costs host time
    # on a path with ~1e5 launches per solve); one extra profiled solve after the
    # timed region gives the per-kernel durations
    cfg = dict(prec=args.prec, eta=args.eta, K=args.K, sparsify_gamma=args.gamma,
               device=local, cuda_stream=stream.cuda_stream, profile=0)
    h = pins.Pins(**cfg)
    res = pins.pins_result()

    def step():
        st = pins.pins_solve(h.h, pdev.prob, res)
        if st not in (0, 3):
            raise RuntimeError(f"pins_solve: {pins.STATUS_NAMES.get(st)}: {h.error()}")
        return res.as_dict()

    for _ in range(args.warmup):
        step()
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    cg_iters = 0
    with ClockSampler(local) as clk:
        flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        ev0.record(stream)
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()                 # L2 flush between timed steps
            out = step()
            launches += out["gpu_launches"]
            cg_iters += out["cg_iters"]
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    value, t = whole_job_rate(ev0.elapsed_time(ev1) / 1e3, args.steps, world, device="cuda")
    # e2e: host pinned inputs -> public API -> potentials back, every step
    hp = {"C": torch.from_numpy(C32).pin_memory(), "a": torch.from_numpy(w.a).pin_memory(),
          "b": torch.from_numpy(w.b).pin_memory()}
    phost = pins.make_problem("dense", hp["a"].numpy(), hp["b"].numpy(), C=hp["C"].numpy())
    Fh = torch.zeros(args.n, dtype=torch.float64).pin_memory()
    Gh = torch.zeros(args.n, dtype=torch.float64).pin_memory()
    r2 = pins.pins_result()
    r2.F_out, r2.G_out = Fh.data_ptr(), Gh.data_ptr()
    e2e_steps = max(1, min(args.steps, 2))
    torch.cuda.synchronize()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        pins.pins_solve(h.h, phost.prob, r2)
    te = time.perf_counter() - te
    h2d = C32.nbytes + w.a.nbytes + w.b.nbytes
    d2h = 2 * args.n * 8
    last = out
    h.close()
    # one profiled solve: per-kernel-class CUDA-event durations
    hp = pins.Pins(**dict(cfg, profile=1))
    rp = pins.pins_result()
    pins.pins_profile_read(hp.h, reset=True)
    pins.pins_solve(hp.h, pdev.prob, rp)
    torch.cuda.synchronize()
    prof = pins.pins_profile_read(hp.h, reset=True)
    prof_cg_iters = rp.as_dict()["cg_iters"]
    hp.close()
    # plain FP64 GPU PINS on the same instance (comparison key)
    fp64 = None
    if args.prec == "mixed" and args.fp64_steps > 0:
        C64d = torch.from_numpy(w.dense_cost()).cuda()
        p64 = pins.make_problem("dense", ad, bd, C=C64d, on_device=True)
        h64 = pins.Pins(prec="fp64", eta=args.eta, K=args.K, sparsify_gamma=args.gamma,
                        device=local, cuda_stream=stream.cuda_stream)
        r64 = pins.pins_result()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.fp64_steps):
            pins.pins_solve(h64.h, p64.prob, r64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64 = e0.elapsed_time(e1) / 1e3 / args.fp64_steps
        d64 = r64.as_dict()
        fp64 = {"value": 1.0 / t64, "unit": "solves/s", "cost": d64["cost"],
                "rel_gap": d64["rel_gap"], "marg_resid_l1": d64["marg_resid_l1"],
                "rel_cost_diff_mixed_vs_fp64": abs(last["cost"] - d64["cost"]) / abs(d64["cost"])}
        h64.close()
    if rank != 0:
        return
    peaks = measured_peaks()
    line = {"metric": "OT solves/s", "value": value, "unit": "solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+dd" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": config_dict(args, w),
            "accuracy": {"cost": last["cost"], "cost_ub": last["cost_ub"],
                         "dual_lb": last["dual_lb"], "certified_rel_gap": last["rel_gap"],
                         "marg_resid_l1": last["marg_resid_l1"],
                         "outer_iters": last["outer_iters"],
                         "sinkhorn_iters": last["sinkhorn_iters"],
                         "newton_iters": last["newton_iters"], "cg_iters": last["cg_iters"]},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": {"value": e2e_steps / te, "unit": "solves/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h},
            "fp64_gpu": fp64,
            "peaks_source": "MEASURED_PEAKS.json" if peaks else "fallback"}
    keep = int(min(args.n * args.n, max(1, round(args.gamma * (2 * args.n - 1)))))
    roof, dom = roofline(prof, args.n, args.n, 4 if args.prec == "mixed" else 8, prof_cg_iters,
                         keep, peaks, args.prec == "mixed")
    if roof is not None:
        if args.prec == "mixed" and args.n == 4096:
            roof["traffic"] = NCU_TRAFFIC_BYTES.get(dom)
            if roof["traffic"] is not None:
                roof["traffic_unit"] = "bytes per launch (ncu, cold caches)"
        roof["timing"] = ("CUDA events on the solver's stream around every launch, one profiled "
                          "solve after the timed region")
    line["roofline"] = roof
    tot = sum(v[0] for v in prof.values()) or 1.0
    line["kernel_time_share"] = {k: round(v[0] / tot, 4) for k, v in prof.items() if v[1]}
    if world == 1:
        line["cpu_baseline"] = cpu_baseline_sample(args, w)
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# serving stream (separate mode, not the contract line)
# --------------------------------------------------------------------------- #
def run_serving(args):
    """Requests of point-cloud pairs (n log-uniform in [nmin, nmax], GMM points,
    Dirichlet(1) weights, certified-gap target 1e-6, paper-default caps) arrive as
    a Poisson stream.  Mixed arm: pins_submit at each arrival time on one handle
    (max_inflight concurrent solves, device-memory admission), completions found
    with pins_poll.  FP64 arm: the same requests solved one at a time in arrival
    order (FIFO).  Latency = completion - arrival."""
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    R = args.serve_requests
    reqs = [wl.serving_request(i, eta=args.eta, n_min=args.serve_nmin, n_max=args.serve_nmax)
            for i in range(R)]
    refs = [pins.problem_from_workload(w) for w in reqs]
    arr = wl.poisson_arrivals(args.serve_rate, R)
    arr = arr - arr[0]
    common = dict(eta=args.eta, K=args.K, tol_gap=1e-6, gap_every=10)
    # warm-up (module load, first-touch allocations)
    hw = pins.Pins(prec="mixed", **common)
    hw.solve(pins.problem_from_workload(wl.serving_request(10**6, eta=args.eta, n_min=256, n_max=256)))
    hw.close()
    h = pins.Pins(prec="mixed", max_inflight=args.serve_inflight, **common)
    done = {}
    pending = {}
    t0 = time.perf_counter()
    k = 0
    while len(done) < R:
        now = time.perf_counter() - t0
        while k < R and arr[k] <= now:
            pending[h.submit(refs[k])] = k
            k += 1
        for t in list(pending):
            d = h.poll(t)
            if d is not None:
                done[pending.pop(t)] = (time.perf_counter() - t0, d)
        time.sleep(0.0005)
    h.close()
    lat = np.array([done[i][0] - arr[i] for i in range(R)])
    span = max(v[0] for v in done.values())
    gaps = [done[i][1]["rel_gap"] for i in range(R)]
    nf = R if args.serve_fp64 < 0 else min(R, args.serve_fp64)
    h64 = pins.Pins(prec="fp64", **common)
    finish, t_prev, solve_s = [], 0.0, []
    for i in range(nf):
        torch.cuda.synchronize()
        ts = time.perf_counter()
        h64.solve(refs[i], want_potentials=False)
        dt = time.perf_counter() - ts
        solve_s.append(dt)
        t_prev = max(t_prev, arr[i]) + dt
        finish.append(t_prev)
    h64.close()
    lat64 = np.array([finish[i] - arr[i] for i in range(nf)]) if nf else np.zeros(1)
    ns = [r.prob.n for r in refs]
    line = {"mode": "serving", "metric": "OT solves/s + p50/p99 latency", "unit": "solves/s",
            "requests": R, "rate_per_s": args.serve_rate,
            "n_range": [args.serve_nmin, args.serve_nmax], "n_median": float(np.median(ns)),
            "config": {"eta": args.eta, "K": args.K, "T1": 100, "T2": 50, "tol_gap": 1e-6,
                       "points": "8-component 2-D GMM, Dirichlet(1) weights, cost /max",
                       "max_inflight": args.serve_inflight},
            "mixed_served": {"solves_per_s": R / span, "p50_s": float(np.percentile(lat, 50)),
                             "p99_s": float(np.percentile(lat, 99)), "makespan_s": span,
                             "median_rel_gap": float(np.median(gaps))},
            "fp64_one_at_a_time": None if nf == 0 else {"requests": nf, "solves_per_s": nf / finish[-1],
                                   "p50_s": float(np.percentile(lat64, 50)),
                                   "p99_s": float(np.percentile(lat64, 99)),
                                   "mean_solve_s": float(np.mean(solve_s))}}
    print(json.dumps(line), flush=True)


def run_batch(args):
    """P stroke-histogram pairs (1-3 thick polylines, shifted or rotated, grids
    drawn from 16^2 ... 64^2, squared pixel distance / max) solved by one
    pins_solve_batch call (instances run concurrently, batch_inflight at a time),
    against plain FP64 PINS one pair at a time within a time budget."""
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    P = args.batch
    refs = [pins.problem_from_workload(wl.stroke_pair(i, eta=args.eta)) for i in range(P)]
    common = dict(eta=args.eta, K=args.K)
    hw = pins.Pins(prec="mixed", **common)
    hw.solve(refs[0]); hw.close()                    # warm-up
    h = pins.Pins(prec="mixed", max_inflight=args.batch_inflight, **common)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs = h.solve_batch(refs)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    h.close()
    h64 = pins.Pins(prec="fp64", **common)
    n64, t64, diffs = 0, 0.0, []
    for i in range(P):
        if t64 > args.fp64_seconds:
            break
        ts = time.perf_counter()
        d = h64.solve(refs[i], want_potentials=False)
        t64 += time.perf_counter() - ts
        n64 += 1
        diffs.append(abs(outs[i]["cost"] - d["cost"]) / abs(d["cost"]))
    h64.close()
    sizes = [r.prob.n for r in refs]
    line = {"mode": "batch", "metric": "OT solves/s", "unit": "solves/s", "pairs": P,
            "grid_sizes": sorted(set(sizes)), "config": {"eta": args.eta, "K": args.K,
                                                         "inflight": args.batch_inflight},
            "mixed_batch": {"solves_per_s": P / tb, "seconds": tb},
            "fp64_one_at_a_time": {"pairs": n64, "solves_per_s": n64 / t64 if t64 else None,
                                   "max_rel_cost_diff_vs_mixed": max(diffs) if diffs else None}}
    print(json.dumps(line), flush=True)


def run_lse_roofline(args):
    """Times the mixed Sinkhorn half-steps (one row and one column pass per
    iteration, each reading the dense FP32 C once) with the library's per-class
    CUDA events, and reports achieved GB/s against the measured HBM copy rate."""
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    n = args.lse_roofline
    w = wl.gmm_instance(0, m=n, n=n, eta=args.eta)
    C = torch.from_numpy(w.dense_cost().astype(np.float32)).cuda()
    a = torch.from_numpy(w.a).cuda(); b = torch.from_numpy(w.b).cuda()
    prob = pins.make_problem("dense", a, b, C=C, on_device=True)
    h = pins.Pins(prec="mixed", eta=args.eta, profile=1)
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    G = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = 50.0                                   # a mid-solve scale s/eta
    pins.pins_step_sinkhorn(h.h, prob.prob, s, 3, F, G, None)      # warm-up
    torch.cuda.synchronize()
    pins.pins_profile_read(h.h, reset=True)
    iters = max(3, args.steps * 5)
    pins.pins_step_sinkhorn(h.h, prob.prob, s, iters, F, G, None)
    torch.cuda.synchronize()
    prof = pins.pins_profile_read(h.h, reset=True)
    h.close()
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    out = {"mode": "lse_roofline", "n": n, "bytes_per_pass": 4 * n * n, "iterations": iters}
    for k in ("row_lse", "col_lse"):
        ms, cnt = prof[k]
        t = ms / cnt / 1e3
        gbs = 4.0 * n * n / t / 1e9
        out[k] = {"us_per_pass": t * 1e6, "achieved_gbs": gbs, "peak_gbs": peak,
                  "frac": gbs / peak}
    print(json.dumps(out), flush=True)


def main():
    args = parse()
    if args.lse_roofline:
        run_lse_roofline(args)
        return
    if args.batch:
        run_batch(args)
        return
    if args.serving:
        run_serving(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
