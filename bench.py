"""Benchmark: served OT solves/s with p50/p99 latency at a certified relative cost
error <= 1e-6 on one GB300, mixed precision served against plain FP64 one at a
time (PINS, Algorithm 2).

Default workload: a served stream of stroke-image pairs -- the shapes of the
paper's augmented-MNIST family (Section 5.1.1): 1-3 thick polylines, shifted or
rotated, on grids drawn uniformly from 16^2 ... 64^2, squared pixel distance
normalised to max 1, the cost generated from grid indices and never stored.
Every request asks for a certified relative gap <= 1e-6 (eta = 2.5e-4, K <= 250,
sparsify budget 2 (m + n - 1)); a request counts as solved only when its
certificate meets the target.  One step = one stream of R requests arriving as
a Poisson process, admitted into the library's serving pool (continuous
batching: requests start as slots and device memory free up, their kernels
overlap on the device).  `value` = certified solves / second over the timed
steps with inputs resident on the device; `e2e` = the same stream through the
public API from pinned host buffers with the potentials read back.

Sub-objects: the same requests solved by plain FP64 PINS one at a time (FIFO at
the same arrival times) beside the mixed served arm on that subset; an
arrival-rate sweep (where saturation begins); the HBM roofline of the mixed
Sinkhorn passes on a stored 16384^2 FP32 cost (1 GiB, beyond L2); the roofline
of the dominant kernel class of a profiled solve; the oracle timed on full
solves of the stream's smallest requests.

Other modes: --workload gmm4096 (one dense 4096^2 GMM instance, the previous
headline), --lse-roofline N, --batch P.  `--impl reference` times the FP64 CPU
oracle on the same workload.
"""
from __future__ import annotations

import os

# the oracle legs run single-threaded (the paper's setting); no effect on the GPU path
for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
# one hardware work queue per serving slot: with the runtime's default of 8
# queues, the pool's 16 solver streams share queues and a short request waits
# behind the kernels of a long one (process-local; read when CUDA starts)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

import argparse  # noqa: E402
import json  # noqa: E402
import subprocess  # noqa: E402
import sys  # noqa: E402
import threading  # noqa: E402
import time  # noqa: E402

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

TOL_GAP = 1e-6


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="strokes", choices=["strokes", "gmm4096"])
    ap.add_argument("--eta", type=float, default=None,
                    help="default 2.5e-4 (strokes), 1e-2 (gmm4096)")
    ap.add_argument("--K", type=int, default=250)
    ap.add_argument("--gamma", type=float, default=None,
                    help="sparsify budget multiplier: default 2 (strokes), 1 (gmm4096)")
    ap.add_argument("--requests", type=int, default=24, help="requests per stream (one step)")
    ap.add_argument("--rate", type=float, default=100.0,
                    help="Poisson arrival rate of the headline stream (req/s)")
    ap.add_argument("--inflight", type=int, default=16, help="serving slots (max_inflight)")
    ap.add_argument("--sweep", default="0.5,1,2,4",
                    help="arrival rates of the saturation sweep ('' to skip)")
    ap.add_argument("--sweep-requests", type=int, default=16)
    ap.add_argument("--fp64-compare", type=int, default=1,
                    help="1: the FP64 one-at-a-time arm on one request per grid size")
    ap.add_argument("--hbm-roofline", type=int, default=16384, metavar="N",
                    help="size of the stored-cost HBM roofline sub-object (0: skip)")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--cpu-all-cores", type=int, default=1,
                    help="1: also time the oracle on every host core (a process pool)")
    # other modes
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--n", type=int, default=4096)
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--lse-roofline", type=int, default=0, metavar="N",
                    help="instead of the contract line: HBM roofline of the mixed Sinkhorn "
                         "passes on an N x N dense FP32 GMM cost")
    ap.add_argument("--batch", type=int, default=0, metavar="P",
                    help="instead of the contract line: P stroke pairs through pins_solve_batch")
    ap.add_argument("--batch-inflight", type=int, default=8)
    ap.add_argument("--single", type=int, default=0, metavar="S",
                    help="instead of the contract line: one mixed solve of the first stroke pair "
                         "on an S x S grid (a warm-up solve first); the command the kernel "
                         "profiles under profiles/ capture")
    ap.add_argument("--fp64-seconds", type=float, default=120.0)
    ap.add_argument("--grids", default="", metavar="S,...",
                    help="instead of the contract line: one mixed solve of the bump-histogram "
                         "instance on each S x S grid (cost generated on the fly), with the "
                         "device memory the solve holds")
    ap.add_argument("--grid-line", type=int, default=64, metavar="S",
                    help="grid size of the default line's bump-histogram sub-object (0: skip)")
    a = ap.parse_args()
    if a.eta is None:
        a.eta = 2.5e-4 if a.workload == "strokes" else 1e-2
    if a.gamma is None:
        a.gamma = 2.0 if a.workload == "strokes" else 1.0
    return a


def whole_job_rate(t_local: float, steps: int, world: int, device: str = "cpu"):
    """Max over ranks of the timed-region length, and the whole-job rate (every
    rank ran `steps` units).  Needs an initialised process group when world > 1
    (NCCL with device='cuda' in the benchmark, gloo with 'cpu' in tests)."""
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


# --------------------------------------------------------------------------- #
# roofline of the dominant kernel class
# --------------------------------------------------------------------------- #
# kernel classes that stream the m x n matrix once per launch
MN_CLASSES = ("row_lse", "col_lse", "marginals", "trial", "key_hist", "key_compact",
              "csr_write", "certificate")
SMS, FP32_LANES, MUFU_PER_SM, SM_GHZ = 152, 128, 16, 2.07
FP32_PEAK_TFLOPS = SMS * FP32_LANES * 2 * SM_GHZ * 1e9 / 1e12     # FMA = 2 flops
EX2_PEAK_GPS = SMS * MUFU_PER_SM * SM_GHZ                          # G ex2 per second
# dram__bytes_read.sum + dram__bytes_write.sum per launch from one ncu capture of
# the class's kernel on the roofline's workload (profiles/); remove an entry
# once its kernel changes after the capture.
NCU_TRAFFIC_BYTES = {
    "cg": 663552 + 0,        # k_pcg_dd, 64 x 64 stroke pair (profiles/k_pcg_dd_stroke64.md)
}


def roofline(prof, m, n, elem_bytes, cg_iters, nnz, peaks, streamed):
    """Roofline object for the class with the largest device time.

    CG (the mixed double-float kernel): the method's own work per iteration,
    4 nnz + 14 (m + n) flops (off-diagonal SpMV on the CSR and CSC copies, the
    diagonal, three inner products and four vector updates), against the FP32
    rate of the units that execute it (152 SMs x 128 lanes x 2 x 2.07 GHz).
    m x n passes on a stored cost: m n elem_bytes algorithmic bytes per launch
    against the measured HBM copy rate.  m x n passes on a streamed cost (grid
    or points, no bytes per entry): entries per second against the MUFU ex2
    rate (152 SMs x 16 per clock x 2.07 GHz), one exponential per entry."""
    dom, (ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    if cnt == 0:
        return None, dom
    t = ms / cnt / 1e3
    if dom == "cg":
        iters = cg_iters / max(cnt, 1)
        per_launch = (4.0 * nnz + 14.0 * (m + n)) * iters
        achieved = per_launch / t / 1e12
        return {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": FP32_PEAK_TFLOPS,
                "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": NCU_TRAFFIC_BYTES.get(dom),
                "peak_source": "derived: FP32 units x clock (152 x 128 x 2 x 2.07 GHz)",
                "work": "4 nnz + 14 (m + n) flops per CG iteration (the method's own work)",
                "avg_launch_us": t * 1e6, "launches": cnt, "iters_per_launch": iters,
                "note": "latency-bound: one exchange (pushed into the replicas) and one cluster barrier per CG iteration"}, dom
    if streamed:
        per_launch = float(m) * n
        achieved = per_launch / t / 1e9
        return {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": EX2_PEAK_GPS,
                "unit": "G entries/s", "frac": achieved / EX2_PEAK_GPS, "traffic": None,
                "peak_source": "derived: MUFU ex2 units x clock (152 x 16 x 2.07 GHz)",
                "avg_launch_us": t * 1e6, "launches": cnt}, dom
    per_launch = float(m) * n * elem_bytes
    peak = peaks.get("hbm_gbs", 6800.0)
    achieved = per_launch / t / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": NCU_TRAFFIC_BYTES.get(dom),
            "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
            "avg_launch_us": t * 1e6, "launches": cnt}, dom


# --------------------------------------------------------------------------- #
# the served stroke stream
# --------------------------------------------------------------------------- #
def stroke_requests(count, eta, offset=0):
    from paper_2502_03749_gb300 import workloads as wl
    return [wl.stroke_pair(offset + i, eta=eta) for i in range(count)]


def one_per_size(eta, limit=64):
    """The first stroke pair of each grid size (16, 28, 32, 48, 64), by instance."""
    from paper_2502_03749_gb300 import workloads as wl
    seen, out = set(), []
    for i in range(limit):
        w = wl.stroke_pair(i, eta=eta)
        if w.grid[0] not in seen:
            seen.add(w.grid[0])
            out.append(w)
    return sorted(out, key=lambda w: w.grid[0])


def solver_cfg(args, prec, **kw):
    return dict(prec=prec, eta=args.eta, K=args.K, tol_gap=TOL_GAP,
                sparsify_gamma=args.gamma, **kw)


def serve_stream(h, refs, arrivals, potentials=None):
    """Submits refs[k] at arrivals[k] seconds after the start, polls until all are
    done.  Returns (latencies, makespan, results)."""
    from paper_2502_03749_gb300 import pins
    R = len(refs)
    done, pending = {}, {}
    t0 = time.perf_counter()
    k = 0
    while len(done) < R:
        now = time.perf_counter() - t0
        while k < R and arrivals[k] <= now:
            pending[h.submit(refs[k])] = k
            k += 1
        for t in list(pending):
            i = pending[t]
            d = h.poll(t, potentials[i] if potentials else None)
            if d is not None:
                done[pending.pop(t)] = (time.perf_counter() - t0, d)
        if k < R and not pending:
            time.sleep(max(0.0, min(arrivals[k] - (time.perf_counter() - t0), 0.002)))
        else:
            time.sleep(0.0002)
    lat = np.array([done[i][0] - arrivals[i] for i in range(R)])
    span = max(v[0] for v in done.values())
    return lat, span, [done[i][1] for i in range(R)]


def certified(res):
    from paper_2502_03749_gb300 import pins
    return res["status"] == pins.PINS_OK and res["rel_gap"] <= TOL_GAP


def fifo_fp64(args, refs, arrivals, local):
    """Plain FP64 PINS one request at a time in arrival order (FIFO)."""
    import torch
    from paper_2502_03749_gb300 import pins
    h = pins.Pins(**solver_cfg(args, "fp64", device=local))
    finish, t_prev, solve_s, outs = [], 0.0, [], []
    try:
        h.solve(refs[0], want_potentials=False)          # warm-up
        for i, r in enumerate(refs):
            torch.cuda.synchronize()
            ts = time.perf_counter()
            d = h.solve(r, want_potentials=False)
            dt = time.perf_counter() - ts
            solve_s.append(dt)
            outs.append(d)
            t_prev = max(t_prev, arrivals[i]) + dt
            finish.append(t_prev)
    finally:
        h.close()
    lat = np.array([finish[i] - arrivals[i] for i in range(len(refs))])
    ok = sum(certified(d) for d in outs)
    return {"requests": len(refs), "certified": ok, "solves_per_s": ok / finish[-1],
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "mean_solve_s": float(np.mean(solve_s)),
            "max_rel_gap": float(max(d["rel_gap"] for d in outs))}, outs


def served_arm(args, refs, arrivals, local, potentials=None):
    from paper_2502_03749_gb300 import pins
    h = pins.Pins(**solver_cfg(args, "mixed", device=local, max_inflight=args.inflight))
    try:
        lat, span, outs = serve_stream(h, refs, arrivals, potentials)
    finally:
        h.close()
    ok = sum(certified(d) for d in outs)
    return {"requests": len(refs), "certified": ok, "solves_per_s": ok / span,
            "p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
            "makespan_s": span, "max_rel_gap": float(max(d["rel_gap"] for d in outs))}, outs


def oracle_sample(args, seconds):
    """Full oracle solves (same settings) of the stream's 16 x 16 requests, one
    after another until the time budget is spent (at least one)."""
    from oracle import pins_oracle as po
    from paper_2502_03749_gb300 import workloads as wl
    small = [w for w in (wl.stroke_pair(i, eta=args.eta) for i in range(64)) if w.grid[0] == 16]
    t0 = time.perf_counter()
    done, gaps = 0, []
    for w in small:
        r = po.pins(w.dense_cost(), w.a, w.b, eta=args.eta, K=args.K, tol_gap=TOL_GAP,
                    gamma=args.gamma)
        done += 1
        gaps.append(r["rel_gap"])
        if time.perf_counter() - t0 > seconds:
            break
    dt = time.perf_counter() - t0
    return done, dt, max(gaps)


def _oracle_solve(idx, eta, K, gamma):
    """One full oracle solve of the idx-th 16 x 16 stroke request (a pool task)."""
    from oracle import pins_oracle as po
    from paper_2502_03749_gb300 import workloads as wl
    small = [w for w in (wl.stroke_pair(i, eta=eta) for i in range(64)) if w.grid[0] == 16]
    w = small[idx % len(small)]
    r = po.pins(w.dense_cost(), w.a, w.b, eta=eta, K=K, tol_gap=TOL_GAP, gamma=gamma)
    return r["rel_gap"]


def oracle_sample_cores(args, seconds, cores):
    """The same oracle solves, one per host core at a time (a spawn-started process
    pool, one BLAS thread each), until the time budget is spent (at least one
    round).  Returns (solves, seconds, max gap)."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    with ctx.Pool(cores) as pool:
        # warm the workers (imports) outside the timed region
        pool.starmap(_oracle_solve, [(i, args.eta, 1, args.gamma) for i in range(cores)])
        t0 = time.perf_counter()
        done, gmax, k = 0, 0.0, 0
        while True:
            gaps = pool.starmap(_oracle_solve,
                                [(k + i, args.eta, args.K, args.gamma) for i in range(cores)])
            k += cores
            done += len(gaps)
            gmax = max(gmax, max(gaps))
            if time.perf_counter() - t0 > seconds:
                break
        dt = time.perf_counter() - t0
    return done, dt, gmax


def cpu_model():
    """The host CPU's model name, as the OS reports it."""
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=5).stdout
        for line in out.splitlines():
            if line.strip().lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.machine()


def run_ours_strokes(args):
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    rank, world, local = dist_info()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    torch.cuda.set_device(local)
    R = args.requests
    ws = stroke_requests(R, args.eta)
    arrivals = wl.poisson_arrivals(args.rate, R)
    arrivals = arrivals - arrivals[0]
    # inputs resident on the device: the marginals (the grid cost needs no array)
    dev_refs = [pins.make_problem("grid", torch.from_numpy(w.a).cuda(),
                                  torch.from_numpy(w.b).cuda(), cost_scale=w.cost_scale,
                                  grid=w.grid, on_device=True) for w in ws]
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    # one serving handle for the warm-up and timed steps: its workers keep their
    # arenas (device-memory admission still applies), as a long-running server does
    h = pins.Pins(**solver_cfg(args, "mixed", device=local, max_inflight=args.inflight))
    for _ in range(args.warmup):
        serve_stream(h, dev_refs, arrivals)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lats, outs_all, certified_total, t_dev = [], [], 0, 0.0
    with ClockSampler(local) as clk:
        for _ in range(args.steps):
            flush.zero_()                       # L2 flush between timed steps
            torch.cuda.synchronize()
            ev0.record()
            lat, span, outs = serve_stream(h, dev_refs, arrivals)
            torch.cuda.synchronize()
            ev1.record()
            torch.cuda.synchronize()
            t_dev += ev0.elapsed_time(ev1) / 1e3
            lats.extend(lat.tolist())
            outs_all.extend(outs)
            certified_total += sum(certified(d) for d in outs)
    if world > 1:
        torch.distributed.barrier()
    rate_steps, t = whole_job_rate(t_dev, args.steps, world, device="cuda")
    value = rate_steps * certified_total / args.steps
    launches = int(sum(d["gpu_launches"] for d in outs_all))
    # e2e: host (pinned) marginals submitted through the public API, potentials read back
    host = []
    for w in ws:
        a = torch.from_numpy(w.a).pin_memory()
        b = torch.from_numpy(w.b).pin_memory()
        host.append((a, b))
    host_refs = [pins.make_problem("grid", host[i][0].numpy(), host[i][1].numpy(),
                                   cost_scale=w.cost_scale, grid=w.grid) for i, w in enumerate(ws)]
    pots = [(torch.zeros(w.m, dtype=torch.float64).pin_memory().numpy(),
             torch.zeros(w.n, dtype=torch.float64).pin_memory().numpy()) for w in ws]
    te, e2e_ok = 0.0, 0
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ts = time.perf_counter()
        _, _, outs = serve_stream(h, host_refs, arrivals, pots)
        te += time.perf_counter() - ts
        e2e_ok += sum(certified(d) for d in outs)
    h.close()
    h2d = int(sum(w.a.nbytes + w.b.nbytes for w in ws))
    d2h = int(sum(8 * (w.m + w.n) for w in ws))
    if rank != 0:
        return
    peaks = measured_peaks()
    gaps = np.array([d["rel_gap"] for d in outs_all])
    line = {"metric": "OT solves/s + p50/p99 latency at rel cost err <= 1e-6, served vs plain FP64",
            "value": value, "unit": "certified solves/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+dd", "data": "synthetic",
            "config": {"workload": f"served stream of {R} stroke-image pairs per step "
                                   "(1-3 thick polylines, shifted/rotated, grids drawn from "
                                   "16^2..64^2, squared pixel distance / max, cost from grid "
                                   f"indices), Poisson arrivals at {args.rate:g}/s, each "
                                   f"certified to rel gap <= {TOL_GAP:g}",
                       "eta": args.eta, "K": args.K, "T1": 100, "T2": 50,
                       "sparsify_gamma": args.gamma, "tol_gap": TOL_GAP,
                       "max_inflight": args.inflight, "precision": "mixed (FP32 + double-float)",
                       "grid_sizes": [w.grid[0] for w in ws],
                       "l2_note": "grid costs are generated, not stored; L2 flushed (256 MiB "
                                  "write) between timed steps",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "cuda_device_max_connections": os.environ.get("CUDA_DEVICE_MAX_CONNECTIONS")},
            "latency": {"p50_s": float(np.percentile(lats, 50)),
                        "p99_s": float(np.percentile(lats, 99)),
                        "of": "completion - arrival, every timed request"},
            "accuracy": {"requests": len(outs_all), "certified": certified_total,
                         "max_rel_gap": float(gaps.max()), "median_rel_gap": float(np.median(gaps)),
                         "statuses": sorted({int(d["status"]) for d in outs_all})},
            "gpu_launches": launches,
            "clocks": clk.summary(),
            "e2e": {"value": e2e_ok / te, "unit": "certified solves/s",
                    "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                    "note": "pins_submit from pinned host marginals, potentials read back by "
                            "pins_poll; wall clock over the same number of steps"},
            "peaks_source": "MEASURED_PEAKS.json" if peaks else "fallback"}
    # like-for-like: one request per grid size, both arms on the same arrivals
    if args.fp64_compare:
        sub = one_per_size(args.eta)
        sub_refs = [pins.problem_from_workload(w) for w in sub]
        sub_arr = np.zeros(len(sub))
        mixed_sub, mo = served_arm(args, sub_refs, sub_arr, local)
        fp64_sub, fo = fifo_fp64(args, sub_refs, sub_arr, local)
        diffs = [abs(a["cost"] - b["cost"]) / abs(b["cost"]) for a, b in zip(mo, fo)]
        line["fp64_compare"] = {
            "requests": "first stroke pair of each grid size " + str([w.grid[0] for w in sub]) +
                        ", all arriving at t = 0",
            "mixed_served": mixed_sub, "fp64_one_at_a_time": fp64_sub,
            "speedup_solves_per_s": mixed_sub["solves_per_s"] / fp64_sub["solves_per_s"],
            "max_rel_cost_diff": float(max(diffs))}
    # saturation sweep
    if args.sweep:
        sweep = []
        sw = stroke_requests(args.sweep_requests, args.eta, offset=1000)
        sw_refs = [pins.problem_from_workload(w) for w in sw]
        for lam in [float(x) for x in args.sweep.split(",") if x]:
            arr = wl.poisson_arrivals(lam, len(sw), instance=int(lam * 1000))
            arr = arr - arr[0]
            d, _ = served_arm(args, sw_refs, arr, local)
            sweep.append({"rate_per_s": lam, "solves_per_s": d["solves_per_s"],
                          "p50_s": d["p50_s"], "p99_s": d["p99_s"], "certified": d["certified"]})
        line["rate_sweep"] = {"requests_per_rate": len(sw), "points": sweep}
    # profiled solve of a 64 x 64 request: per-class device time and the roofline
    big = next(w for w in ws if w.grid[0] == 64)
    hp = pins.Pins(**solver_cfg(args, "mixed", device=local, profile=1))
    pins.pins_profile_read(hp.h, reset=True)
    rp = hp.solve(pins.problem_from_workload(big), want_potentials=False)
    torch.cuda.synchronize()
    prof = pins.pins_profile_read(hp.h, reset=True)
    hp.close()
    keep = int(round(args.gamma * (big.m + big.n - 1)))
    roof, dom = roofline(prof, big.m, big.n, 4, rp["cg_iters"], keep, peaks, streamed=True)
    if roof is not None:
        roof["workload"] = "one 64 x 64 stroke pair of the stream, profiled solve"
        roof["timing"] = ("CUDA events on the solver's stream around every launch, one "
                          "profiled solve after the timed region")
    line["roofline"] = roof
    tot = sum(v[0] for v in prof.values()) or 1.0
    line["kernel_time_share"] = {k: round(v[0] / tot, 4) for k, v in prof.items() if v[1]}
    if args.hbm_roofline:
        line["hbm_roofline"] = lse_roofline(args, args.hbm_roofline)
    if args.grid_line:
        line["grid_histograms"] = grid_solve(args, args.grid_line)
        line["grid_histograms"]["workload"] = (
            "bump histograms (5-20 Gaussian bumps + 1e-6 floor) on a "
            f"{args.grid_line} x {args.grid_line} grid, squared grid distance / max, "
            "cost generated on the fly")
    if world == 1:
        done, dt, gmax = oracle_sample(args, args.cpu_seconds)
        model = cpu_model()
        line["cpu_baseline"] = {
            "value": done / dt, "unit": "certified solves/s", "cores": 1, "kind": "oracle",
            "cpu": model,
            "sample": f"{done} full oracle solves of the stream's 16 x 16 requests "
                      f"({dt:.1f} s, max rel gap {gmax:.1e}); the stream's larger grids take "
                      "the oracle minutes each, so this favours the oracle"}
        if args.cpu_all_cores:
            cores = os.cpu_count() or 1
            try:
                done, dt, gmax = oracle_sample_cores(args, args.cpu_seconds / 2, cores)
                line["cpu_baseline_all_cores"] = {
                    "value": done / dt, "unit": "certified solves/s", "cores": cores,
                    "kind": "oracle", "cpu": model,
                    "sample": f"{done} full oracle solves of the same requests, one per core "
                              f"at a time ({dt:.1f} s, max rel gap {gmax:.1e})"}
            except Exception as e:   # a host without process pools still prints its line
                line["cpu_baseline_all_cores"] = {"unavailable": f"{type(e).__name__}: {e}"}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# reference arm: the FP64 CPU oracle on the same workload
# --------------------------------------------------------------------------- #
def run_reference(args):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    if args.workload != "strokes":
        print(json.dumps({"impl": "reference", "unavailable":
                          "the oracle arm is timed on the default served stroke workload"}))
        return
    per = max(2.0, args.cpu_seconds / 4)
    for _ in range(args.warmup):
        oracle_sample(args, 0.0)
    t, n, gmax = 0.0, 0, 0.0
    for _ in range(args.steps):
        d, dt, g = oracle_sample(args, per)
        n += d
        t += dt
        gmax = max(gmax, g)
    val = n / t
    line = {"impl": "reference", "metric": "OT solves/s + p50/p99 latency at rel cost err "
                                            "<= 1e-6, served vs plain FP64",
            "value": val, "unit": "certified solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": "the served stroke-pair stream's 16 x 16 requests, solved "
                                   "one at a time by the FP64 CPU oracle to rel gap <= 1e-6",
                       "eta": args.eta, "K": args.K, "sparsify_gamma": args.gamma},
            "cpu_baseline": {"value": val, "unit": "certified solves/s", "cores": 1,
                             "kind": "oracle",
                             "sample": f"{n} full oracle solves over {args.steps} steps "
                                       f"(max rel gap {gmax:.1e})"},
            "e2e": {"value": val, "unit": "certified solves/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------- #
# other modes
# --------------------------------------------------------------------------- #
def lse_roofline(args, n, iters_per_step=5):
    """Mixed Sinkhorn half-steps on a stored N x N FP32 GMM cost (one row and one
    column pass per iteration, each reading C once), timed with the library's
    per-class CUDA events; achieved GB/s against the measured HBM copy rate."""
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    w = wl.gmm_instance(0, m=n, n=n, eta=1e-2, as_dense=False)
    x = torch.from_numpy(w.x).cuda()
    y = torch.from_numpy(w.y).cuda()
    C = (torch.cdist(x, y) ** 2 * w.cost_scale).to(torch.float32).contiguous()
    a = torch.from_numpy(w.a).cuda(); b = torch.from_numpy(w.b).cuda()
    prob = pins.make_problem("dense", a, b, C=C, on_device=True)
    h = pins.Pins(prec="mixed", eta=1e-2, profile=1)
    F = torch.zeros(n, dtype=torch.float64, device="cuda")
    G = torch.zeros(n, dtype=torch.float64, device="cuda")
    s = 50.0
    try:
        pins.pins_step_sinkhorn(h.h, prob.prob, s, 3, F, G, None)
        torch.cuda.synchronize()
        pins.pins_profile_read(h.h, reset=True)
        iters = max(3, args.steps * iters_per_step)
        pins.pins_step_sinkhorn(h.h, prob.prob, s, iters, F, G, None)
        torch.cuda.synchronize()
        prof = pins.pins_profile_read(h.h, reset=True)
    finally:
        h.close()
    del C
    torch.cuda.empty_cache()
    peak = measured_peaks().get("hbm_gbs", 6800.0)
    out = {"n": n, "bytes_per_pass": 4 * n * n, "iterations": iters,
           "cost": "dense FP32 GMM cost (C = 4 n^2 bytes, beyond L2), s/eta = 5e3"}
    for k in ("row_lse", "col_lse"):
        ms, cnt = prof[k]
        t = ms / cnt / 1e3
        gbs = 4.0 * n * n / t / 1e9
        out[k] = {"us_per_pass": t * 1e6, "achieved_gbs": gbs, "peak_gbs": peak,
                  "frac": gbs / peak}
    return out


def run_gmm4096(args):
    """One dense m = n = 4096 GMM instance (Dirichlet(1) weights, eta = 1e-2,
    paper caps): a whole solve per step, FP64 comparison.  This instance does
    not reach a certified 1e-6 within K = 250."""
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    w = wl.gmm_instance(0, m=args.n, n=args.n, eta=args.eta)
    C32 = w.dense_cost().astype(np.float32) if args.prec == "mixed" else w.dense_cost()
    Cd = torch.from_numpy(C32).cuda()
    ad = torch.from_numpy(w.a).cuda()
    bd = torch.from_numpy(w.b).cuda()
    pdev = pins.make_problem("dense", ad, bd, C=Cd, on_device=True)
    stream = torch.cuda.Stream()
    cfg = dict(prec=args.prec, eta=args.eta, K=args.K, sparsify_gamma=args.gamma,
               device=local, cuda_stream=stream.cuda_stream, tol_gap=TOL_GAP, gap_every=10)
    h = pins.Pins(**cfg)
    res = pins.pins_result()
    for _ in range(args.warmup):
        pins.pins_solve(h.h, pdev.prob, res)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        pins.pins_solve(h.h, pdev.prob, res)
    e1.record(stream)
    torch.cuda.synchronize()
    h.close()
    d = res.as_dict()
    t = e0.elapsed_time(e1) / 1e3 / args.steps
    print(json.dumps({"mode": "gmm4096", "solves_per_s": 1.0 / t, "seconds_per_solve": t,
                      "cost": d["cost"], "cost_ub": d["cost_ub"], "dual_lb": d["dual_lb"],
                      "certified_rel_gap": d["rel_gap"], "marg_resid_l1": d["marg_resid_l1"],
                      "outer_iters": d["outer_iters"], "newton_iters": d["newton_iters"],
                      "cg_iters": d["cg_iters"], "eta": args.eta, "gamma": args.gamma}),
          flush=True)


def grid_solve(args, S, prec="mixed", K=None):
    """One solve of the bump-histogram instance on an S x S grid (config 3's
    recipe), certified gap target 1e-6.  Device memory: free memory before the
    handle is created minus free memory after the solve (the handle keeps its
    workspace until closed), so it covers everything the library holds."""
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    w = wl.grid_instance(S, 0, eta=args.eta)
    ref = pins.problem_from_workload(w)
    torch.cuda.synchronize()
    free0, total = torch.cuda.mem_get_info()
    cfg = solver_cfg(args, prec)
    if K is not None:
        cfg["K"] = K
    h = pins.Pins(**cfg)
    try:
        t = time.perf_counter()
        d = h.solve(ref, want_potentials=False)
        torch.cuda.synchronize()
        t = time.perf_counter() - t
        free1, _ = torch.cuda.mem_get_info()
    finally:
        h.close()
    return {"grid": S, "n": w.n, "entries_per_pass": float(w.n) * w.n, "prec": prec,
            "seconds": t, "certified": bool(certified(d)), "rel_gap": d["rel_gap"],
            "outer_iters": d["outer_iters"], "newton_iters": d["newton_iters"],
            "cg_iters": d["cg_iters"], "status": d["status"],
            "device_bytes": int(free0 - free1),
            "dense_cost_bytes_if_stored": 4 * w.n * w.n}


def run_grids(args):
    for S in [int(x) for x in args.grids.split(",") if x]:
        print(json.dumps(dict(mode="grid", eta=args.eta, gamma=args.gamma,
                              **grid_solve(args, S, args.prec, args.K))), flush=True)


def run_batch(args):
    """P stroke pairs solved by one pins_solve_batch call (instances run
    concurrently, batch_inflight at a time), certified to 1e-6."""
    import torch
    from paper_2502_03749_gb300 import pins
    P = args.batch
    refs = [pins.problem_from_workload(w) for w in stroke_requests(P, args.eta)]
    h = pins.Pins(**solver_cfg(args, "mixed", max_inflight=args.batch_inflight))
    h.solve(refs[0])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    outs = h.solve_batch(refs)
    torch.cuda.synchronize()
    tb = time.perf_counter() - t0
    h.close()
    ok = sum(certified(d) for d in outs)
    print(json.dumps({"mode": "batch", "pairs": P, "certified": ok, "solves_per_s": ok / tb,
                      "seconds": tb, "max_rel_gap": max(d["rel_gap"] for d in outs),
                      "inflight": args.batch_inflight}), flush=True)


def run_single(args):
    import torch
    from paper_2502_03749_gb300 import pins, workloads as wl
    w = next(w for w in (wl.stroke_pair(i, eta=args.eta) for i in range(64))
             if w.grid[0] == args.single)
    ref = pins.problem_from_workload(w)
    h = pins.Pins(**solver_cfg(args, args.prec))
    try:
        h.solve(ref, want_potentials=False)
        torch.cuda.synchronize()
        t = time.perf_counter()
        d = h.solve(ref, want_potentials=False)
        torch.cuda.synchronize()
        t = time.perf_counter() - t
    finally:
        h.close()
    print(json.dumps({"mode": "single", "grid": args.single, "prec": args.prec, "seconds": t,
                      "rel_gap": d["rel_gap"], "outer_iters": d["outer_iters"],
                      "newton_iters": d["newton_iters"], "cg_iters": d["cg_iters"],
                      "gpu_launches": d["gpu_launches"]}), flush=True)


def main():
    args = parse()
    if args.single:
        run_single(args)
        return
    if args.lse_roofline:
        print(json.dumps(dict(mode="lse_roofline", **lse_roofline(args, args.lse_roofline))),
              flush=True)
        return
    if args.batch:
        run_batch(args)
        return
    if args.grids:
        run_grids(args)
        return
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "gmm4096":
        run_gmm4096(args)
        return
    run_ours_strokes(args)


if __name__ == "__main__":
    main()
