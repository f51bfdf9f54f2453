"""Benchmark: contour-integral quadrature solves per second on one GB300 (or N replicas).

A step is one whole contour-integral pass over the n = 4096 (64 x 64 grid, bandwidth 64)
delay problem with N = 64 quadrature points, L = 16 probe columns and M = 8 moments:
assembly, banded LU, solves refined to backward error <= 1e-10 (a double-float residual with
complex64 factors), moments, block-Hankel SVD, reduced eigenproblem, Rayleigh-Ritz with
Newton, scaled residuals. `value` counts quadrature solves (one (problem, z_j) pair with all
L columns refined) per second with the operator and V resident in HBM; `e2e` is the same
metric through the request server (nep_create_split, nep_submit with the host probe block,
nep_server_wait returning the pairs on the host), copies included.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision mixed|fp64]
                  [--impl ours|reference] [--workload delay2d_s64]

`--impl reference` times the CPU oracle on this host's cores. Multi-GPU runs (torchrun)
solve independent problems per rank (replicas, weak scaling, no collective on the data path).
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

# 32 hardware work queues instead of CUDA's default 8, set before the first CUDA call: the
# pipelines' and server workers' streams then do not share queues, and a request's short result
# copies do not wait behind another pipeline's pass.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "CISS quadrature solves/s & p99 latency, mixed vs FP64 on GB300 at resid\u22641e-10"
UNIT = "quadrature_solves/s"


def pattern_bandwidths(mats):
    """(kl, ku) of the union sparsity pattern of the A_i (a property of the input, not of the method)."""
    import scipy.sparse as sp
    kl = ku = 0
    for A in mats:
        c = sp.coo_matrix(A)
        if c.nnz:
            d = c.row.astype(np.int64) - c.col.astype(np.int64)
            kl, ku = max(kl, int(d.max())), max(ku, int(-d.min()))
    return kl, ku


def workload_config(name, p):
    """The `config` both arms print for a workload: its sizes and the L2 statement."""
    kl, ku = pattern_bandwidths(p.mats)
    band_mb = p.N * p.n * (2 * kl + ku + 1) * 8 / 1e6
    return {"workload": name, "n": p.n, "bandwidth": kl, "N": p.N, "L": p.L, "M": p.M,
            "l2": f"inputs larger than L2 (the complex64 band alone is {band_mb:.0f} MB per step)"}


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def job_throughput(ms_rank: float, world: int, units_per_step_rank: int, device: str = "cuda"):
    """Whole-job throughput of independent replicas: every rank ran the same number of steps on
    its own problem; the job's step time is the slowest rank's (max over ranks), and the job's
    units are all ranks' units. Returns (ms per step of the job, units per second)."""
    ms = ms_rank
    if world > 1:
        import torch
        import torch.distributed as dist
        t = torch.tensor([ms_rank], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_step_rank / (ms * 1e-3)


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


def lu_flops(n, kl, ku, npts):
    """Algorithmic real flops of the banded LU: n steps x kl rows x (kl+ku) columns x 8 (complex FMA)."""
    return 8.0 * n * kl * (kl + ku) * npts


def solve_flops(n, kl, ku, L, npts):
    """Forward (kl) plus backward (kl+ku) complex FMAs per row and right-hand side, 8 flops each."""
    return 8.0 * n * (2 * kl + ku) * L * npts


def solve_bytes(n, ldab, L, npts, esz):
    """Factor band and pivots read once, right-hand sides read and written once."""
    return npts * (n * ldab * esz + 4 * n + 2 * n * L * esz)


# DRAM bytes (read + write) of one solve launch from an ncu capture of the same launch,
# keyed by (workload, precision); None where no capture of the current kernel exists.
SOLVE_TRAFFIC = {("delay2d_s64", "mixed"): (199.1 + 23.9 + 301.0 + 28.6) * 1e6}


def fp32_alu_peak_tflops(sm_mhz):
    """152 SMs x 128 FP32 lanes x 2 flops (FMA) x clock."""
    return 152 * 128 * 2 * sm_mhz * 1e6 / 1e12


def fp64_alu_peak_tflops(sm_mhz):
    """Measured 1.75 FP64 FMA/clk/SM on this part: 152 x 1.75 x 2 flops x clock."""
    return 152 * 1.75 * 2 * sm_mhz * 1e6 / 1e12


def tf32_peak_tflops(peaks):
    """TF32 dense tensor peak: the measured bf16 burst figure x the nominal TF32/bf16 ratio (1.125/2.25)."""
    return peaks.get("bf16_tflops", 1900.0) * 0.5


def cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform
    return platform.processor() or platform.machine()


def arm_bench(binding, p, prec, V, streams, steps, warmup):
    """Throughput of one workload at one precision: `streams` independent pipelines (a plan, a
    non-blocking stream and a host thread each), `steps` full passes in all, CUDA events around them;
    then one pass alone for the latency and the per-stage device times."""
    import torch
    split = binding.Split.from_problem(p)
    S = max(1, min(streams, steps))
    plans = [binding.Plan(split, p.region, p.N, p.L, p.M, precision=prec) for _ in range(S)]
    strs = [torch.cuda.Stream() for _ in range(S)]
    Vd = torch.from_numpy(np.asfortranarray(V).ravel(order="F").view(np.float64).copy()).cuda()
    for i in range(S):
        for _ in range(max(1, warmup)):
            plans[i].execute(Vd, strs[i].cuda_stream)
    torch.cuda.synchronize()

    def run(i):
        for _ in range(i, steps, S):
            plans[i].execute(Vd, strs[i].cuda_stream)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record()
    for st_ in strs:
        st_.wait_event(e0)
    th = [threading.Thread(target=run, args=(i,)) for i in range(S)]
    for t_ in th:
        t_.start()
    for t_ in th:
        t_.join()
    for st_ in strs:
        ev = torch.cuda.Event()
        ev.record(st_)
        torch.cuda.current_stream().wait_event(ev)
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    plans[0].execute(Vd, strs[0].cuda_stream)
    torch.cuda.synchronize()
    r = plans[0].result()
    info = r["info"]
    out = {"ms_per_step": ms, "value": p.N / (ms * 1e-3), "streams": S, "steps": steps,
           "single_pass_ms": info["ms_total"],
           "stages_ms": {k: info[k] for k in ("ms_assemble", "ms_factor", "ms_solve", "ms_moments", "ms_extract")},
           "result": {"nconv": int(len(r["lam"])), "hankel_rank": r["m"], "max_backward": info["max_backward"],
                      "max_sweeps": info["max_sweeps"], "flags": r["flags"],
                      "max_eta": float(r["eta"].max()) if len(r["eta"]) else None}}
    for pl in plans:
        pl.close()
    split.close()
    return out


def wide_config_bench(binding, name, peaks, streams, steps, rank=0):
    """A wide-band workload (Drude 128x128, bandwidth 128; square root 24^3, bandwidth 576): the
    mixed path (complex64 factors with the tensor-core trailing update, double-float refinement) over
    `streams` pipelines, one plain FP64 pass beside it, and the roofline of its dominant kernel,
    the banded LU: algorithmic flops 8 n kl (kl+ku) per point over the LU's device time against the
    TF32 tensor peak; the tensor work executed is 3x that (the hi/lo split's three products)."""
    import synth
    p = synth.config_problem(name, seed=rank)
    V = synth.random_probe_block(p.n, p.L, rank)
    split = binding.Split.from_problem(p)
    kl, ku = split.kl, split.ku
    split.close()
    mixed = arm_bench(binding, p, binding.NEP_PREC_MIXED, V, streams, steps, 1)
    fp64 = arm_bench(binding, p, binding.NEP_PREC_FP64, V, 1, 1, 1)
    lu_ms = mixed["stages_ms"]["ms_factor"]
    fl = lu_flops(p.n, kl, ku, p.N)
    peak = tf32_peak_tflops(peaks)
    ach = fl / (lu_ms * 1e-3) / 1e12
    return {"workload": name, "n": p.n, "bandwidth": kl, "N": p.N, "L": p.L, "M": p.M,
            "ms_per_step": mixed["ms_per_step"], "value": mixed["value"], "unit": UNIT, "mixed": mixed,
            "fp64": fp64, "mixed_over_fp64": mixed["value"] / fp64["value"],
            "roofline": {"kernel": "lu_tc_kernel (banded LU, trailing update on tcgen05 kind::tf32)", "bound": "tensor",
                         "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                         "executed_tensor_frac": 3 * ach / peak, "traffic": None,
                         "ms_per_launch": lu_ms, "algorithmic_flops": fl,
                         "peak_source": "measured bf16 burst (MEASURED_PEAKS.json) x nominal TF32/bf16 ratio 0.5"}}


def cpu_sample_points(p, npts, threads):
    """The oracle's quadrature solves (assembly, band LU, solves, FP64 refinement) at the first npts
    nodes, with `threads` threads over points; returns solves per second."""
    from oracle import ciss
    import synth
    import concurrent.futures as cf
    from oracle import band, contour
    V = synth.random_probe_block(p.n, p.L, 0)
    z, _, _ = contour.nodes(p.region, p.N)
    F = contour.coefficient_table(p.fns, z)
    kl, ku = band.bandwidths(p.mats)
    t0 = time.perf_counter()
    with cf.ThreadPoolExecutor(threads) as ex:
        list(ex.map(lambda j: ciss.solve_point(p, kl, ku, F[:, j], V), range(npts)))
    return npts / (time.perf_counter() - t0)


def cpu_baseline(p, steps_budget_s=20.0):
    """The oracle as it stands on this host's cores: full passes of the same workload until ~budget."""
    from oracle import ciss
    import synth
    V = synth.random_probe_block(p.n, p.L, 0)
    times = []
    t_end = time.perf_counter() + steps_budget_s
    while True:
        t0 = time.perf_counter()
        ciss.solve(p, V=V)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() > t_end or len(times) >= 3:
            break
    cores = max(1, min(32, os.cpu_count() or 1))
    out = {"value": p.N * len(times) / sum(times), "unit": UNIT, "cores": cores, "kind": "oracle",
           "cpu_model": cpu_model(), "nproc": os.cpu_count(),
           "sample": f"{len(times)} full CPU passes of {p.name} (N={p.N} quadrature solves each), "
                     f"threads over quadrature points, {sum(times):.1f} s total"}
    # one thread: the quadrature solves alone at the first 4 nodes (they are ~all of a pass's time)
    out["one_thread"] = {"value": cpu_sample_points(p, 4, 1), "unit": UNIT,
                         "sample": f"quadrature solves at 4 of the {p.N} nodes of {p.name}, one thread"}
    # the oracle's residual inverse iteration on the same operator: one pair from a seeded start at
    # the region's centre, three iterations without a stopping tolerance (one band LU at sigma, then
    # per iteration the inner Newton loop's solves and the update's)
    from oracle import rii
    x0 = synth.random_probe_block(p.n, 1, 1)[:, 0]
    t0 = time.perf_counter()
    rii.rii(p, complex(p.region["center"]), x0, tol=0.0, max_it=2)
    out["rii_s_per_pair_3_iterations"] = time.perf_counter() - t0
    return out


def serving_bench(binding, prec, count, seed, workers, s_max, loads=(0.5, 0.8, 1.2), max_batch=1, fp64=True):
    """Continuous-batching serving on a bounded sample of the Poisson request stream.

    Requests: the first `count` of the seeded delay/Drude stream (s x s grids, n log-uniform up to
    s_max^2, N in {32,64,128}, L in {8,16,32}, M = 8). Capacity is the request rate of the whole
    sample submitted at once; the stream is then replayed in real time at offered loads rho x
    capacity (Poisson inter-arrival gaps rescaled). Latency = submission to result ready.
    Baseline: plain FP64, one request at a time (a server with one worker), replayed under the same
    arrival times and measured the same way.
    """
    import synth
    reqs = synth.serving_requests(count=count, seed=seed, s_max=s_max)
    probs = [synth.serving_problem(r) for r in reqs]
    splits = [binding.Split.from_problem(p) for p in probs]
    Vs = [synth.random_probe_block(p.n, p.L, r["seed"] % 1000) for p, r in zip(probs, reqs)]
    solves = sum(p.N for p in probs)
    gaps = np.diff([0.0] + [r["arrival"] for r in reqs])
    gaps = gaps / gaps.mean()

    def submit(srv, i, pr):
        p = probs[i]
        return srv.submit(splits[i], p.region, p.N, p.L, p.M, V=Vs[i], precision=pr)

    def replay(srv, rate, pr):
        arrivals = np.cumsum(gaps) / rate
        t0 = time.perf_counter()
        tk = []
        for i in range(count):
            d = arrivals[i] - (time.perf_counter() - t0)
            if d > 0:
                time.sleep(d)
            tk.append(submit(srv, i, pr))
        lat = np.array([srv.wait(t)["info"]["ms_latency"] for t in tk])
        span = time.perf_counter() - t0
        return {"rho": None, "offered_req_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "solves_per_s": solves / span}

    srv = binding.Server(workers=workers, max_batch=max_batch)
    for i in range(min(4, count)):  # warm the allocator pool and the library
        srv.wait(submit(srv, i, prec))
    t0 = time.perf_counter()
    tickets = [submit(srv, i, prec) for i in range(count)]
    for t in tickets:
        srv.wait(t)
    capacity = count / (time.perf_counter() - t0)
    out = {"requests": count, "workers": workers, "max_batch": max_batch,
           "n_range": [min(p.n for p in probs), max(p.n for p in probs)],
           "capacity_req_per_s": capacity, "capacity_solves_per_s": capacity * solves / count, "loads": []}
    for rho in loads:
        r_ = replay(srv, rho * capacity, prec)
        r_["rho"] = rho
        out["loads"].append(r_)
    srv.close()
    if not fp64:
        for sp in splits:
            sp.close()
        out["sample"] = f"first {count} requests of the seeded Poisson request stream (seed {seed})"
        return out
    # plain FP64, one request at a time, under the same arrival times
    srv64 = binding.Server(workers=1)
    srv64.wait(submit(srv64, 0, binding.NEP_PREC_FP64))
    base = {"loads": [], "measured": "a one-worker server in plain FP64, replayed under the same arrivals"}
    for rho in loads:
        r_ = replay(srv64, rho * capacity, binding.NEP_PREC_FP64)
        r_["rho"] = rho
        base["loads"].append(r_)
    srv64.close()
    out["fp64_one_at_a_time"] = base
    out["sample"] = (f"first {count} requests of the seeded Poisson request stream (seed {seed}; the full "
                     "stream is 2000 requests, --serving-requests 2000); loads relative to the measured "
                     "mixed-precision capacity")
    for sp in splits:
        sp.close()
    return out


def torch_sync():
    import torch
    torch.cuda.synchronize()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=96)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="delay2d_s64")
    ap.add_argument("--points", type=int, default=0,
                    help="override the workload's quadrature points (small cases for profiler captures)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-symmetric", action="store_true")
    ap.add_argument("--no-polish", action="store_true")
    ap.add_argument("--no-nleigs", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain FP64 arm on the same workload")
    ap.add_argument("--no-wide", action="store_true", help="skip the bandwidth-128 and -576 workloads")
    ap.add_argument("--streams", type=int, default=8,
                    help="concurrent pipelines in the timed region: one plan, stream and host thread each")
    ap.add_argument("--serving-requests", type=int, default=40)
    ap.add_argument("--serving-smax", type=int, default=128)
    args = ap.parse_args()
    rank, world, local = dist_env()
    import synth
    p = synth.config_problem(args.workload, seed=rank)
    if args.points > 0:
        p.N = args.points

    if args.impl == "reference":
        if rank != 0:
            return 0
        times = []
        from oracle import ciss
        V = synth.random_probe_block(p.n, p.L, 0)
        for _ in range(max(0, args.warmup)):
            ciss.solve(p, V=V)
        for _ in range(args.steps):
            t0 = time.perf_counter()
            ciss.solve(p, V=V)
            times.append(time.perf_counter() - t0)
        val = p.N * len(times) / sum(times)
        cores = max(1, min(32, os.cpu_count() or 1))
        line = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": workload_config(args.workload, p),
                "cpu_baseline": {"value": val, "unit": UNIT, "cores": cores, "kind": "oracle",
                                 "sample": f"{len(times)} full passes of {args.workload}"},
                "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0

    import torch
    import torch.distributed as dist
    from paper_1910_11712_gb300 import binding

    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    binding.load(build_if_missing=True)
    prec = binding.NEP_PREC_MIXED if args.precision == "mixed" else binding.NEP_PREC_FP64
    split = binding.Split.from_problem(p)
    plan = binding.Plan(split, p.region, p.N, p.L, p.M, precision=prec)
    V = synth.random_probe_block(p.n, p.L, rank)
    Vd = torch.from_numpy(np.asfortranarray(V).ravel(order="F").view(np.float64).copy()).cuda()
    stream = torch.cuda.current_stream().cuda_stream
    for _ in range(max(3, args.warmup)):
        plan.execute(Vd, stream)
    torch.cuda.synchronize()
    res = plan.result()

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # S independent pipelines (a plan, a non-blocking stream and a host thread each) share the GPU:
    # one pass leaves most SMs idle during its latency-bound extraction stage, which the other
    # pipelines' assembly, LU and solves fill. Every step is still one full pass of its own.
    S = max(1, args.streams)
    plans = [plan] + [binding.Plan(split, p.region, p.N, p.L, p.M, precision=prec) for _ in range(S - 1)]
    streams = [torch.cuda.Stream() for _ in range(S)]
    for i in range(S):
        for _ in range(max(3, args.warmup)):
            plans[i].execute(Vd, streams[i].cuda_stream)
    torch.cuda.synchronize()

    def run_steps(i):
        for _ in range(i, args.steps, S):
            plans[i].execute(Vd, streams[i].cuda_stream)

    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    lu_ms = []
    stage = {k: 0.0 for k in ("ms_assemble", "ms_factor", "ms_solve", "ms_moments", "ms_extract")}
    launches0 = binding.kernel_launches()
    with ClockSampler(torch.cuda.current_device() if "CUDA_VISIBLE_DEVICES" not in os.environ else local) as clk:
        barrier()
        e0.record()
        for st_ in streams:
            st_.wait_event(e0)
        workers = [threading.Thread(target=run_steps, args=(i,)) for i in range(S)]
        for w_ in workers:
            w_.start()
        for w_ in workers:
            w_.join()
        for st_ in streams:
            ev = torch.cuda.Event()
            ev.record(st_)
            torch.cuda.current_stream().wait_event(ev)
        e1.record()
        barrier()
    launches = binding.kernel_launches() - launches0  # all steps of the timed region
    ms = e0.elapsed_time(e1) / args.steps
    # one pipeline alone: the latency of a step
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record()
    for _ in range(args.steps):
        plan.execute(Vd, stream)
    s1.record()
    torch.cuda.synchronize()
    ms_single = s0.elapsed_time(s1) / args.steps
    for pl in plans[1:]:
        pl.close()
    # per-stage device times (CUDA events recorded on the launching stream inside the plan),
    # from separate passes after the timed region
    for _ in range(3):
        plan.execute(Vd, stream)
        r = plan.result()
        lu_ms.append(r["info"]["ms_factor"])
        for k in stage:
            stage[k] += r["info"][k] / 3
    # dominant kernel of the step (largest share of the launch list): the banded triangular
    # solve, all N points x L right-hand sides in one launch, through the library's step entry
    # point on the plan's factors; CUDA events on the launching stream, one fresh right-hand
    # side block per launch (each larger than L2 together with the factors it streams)
    ab_ptr, _ = plan.buffer("ab")
    ut_ptr, _ = plan.buffer("ut")
    ipiv_ptr, _ = plan.buffer("ipiv")
    cdt = torch.complex64 if prec == binding.NEP_PREC_MIXED else torch.complex128
    reps = 5
    Bs = [torch.randn(p.N * p.L * p.n, dtype=cdt, device="cuda") for _ in range(reps + 1)]
    binding.band_solve_cols(split, p.N, prec, ab_ptr, ut_ptr, ipiv_ptr, p.L, Bs[reps], stream)
    k0, k1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    k0.record()
    for r_ in range(reps):
        binding.band_solve_cols(split, p.N, prec, ab_ptr, ut_ptr, ipiv_ptr, p.L, Bs[r_], stream)
    k1.record()
    torch.cuda.synchronize()
    solve_ms = k0.elapsed_time(k1) / reps
    del Bs
    ms, value = job_throughput(ms, world, p.N)

    # conjugate-symmetric quadrature on the same workload (real operators only): a real probe
    # block, only the N/2 nodes above the real axis solved
    symmetric = None
    if not args.no_symmetric:
        try:
            Vr = np.asfortranarray(np.random.default_rng(rank).standard_normal((p.n, p.L)).astype(np.complex128))
            Vrd = torch.from_numpy(Vr.ravel(order="F").view(np.float64).copy()).cuda()
            plan_s = binding.Plan(split, p.region, p.N, p.L, p.M, precision=prec, symmetric=1)
            for _ in range(3):
                plan_s.execute(Vrd, stream)
            torch.cuda.synchronize()
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record()
            for _ in range(args.steps):
                plan_s.execute(Vrd, stream)
            s1.record()
            torch.cuda.synchronize()
            ms_s = s0.elapsed_time(s1) / args.steps
            rs = plan_s.result()
            symmetric = {"ms_per_step": ms_s, "quadrature_nodes_per_s": p.N / (ms_s * 1e-3),
                         "points_solved_per_step": p.N // 2, "nconv": int(len(rs["lam"])), "hankel_rank": rs["m"],
                         "probe": "real N(0,1)"}
            plan_s.close()
        except binding.NepError as e:
            symmetric = {"unavailable": str(e)}

    # residual inverse iteration (Sec. 4.1, Algorithm rii) on the pairs just returned, to a tighter
    # eta than the contour method's: one assembly + band LU at the P starting eigenvalues, then
    # per iteration one band solve with nterms+1 right-hand sides per pair
    polish = None
    if not args.no_polish:
        try:
            plan.execute(Vd, stream)
            torch.cuda.synchronize()
            before = plan.result()
            tol = 1e-13
            q0, q1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            q0.record()
            npol, its = plan.polish(tol=tol, max_it=10, stream=stream)
            q1.record()
            torch.cuda.synchronize()
            after = plan.result()
            polish = {"tol": tol, "pairs": int(npol), "iterations": int(its), "ms": q0.elapsed_time(q1),
                      "max_eta_before": float(before["eta"].max()) if len(before["eta"]) else None,
                      "max_eta_after": float(after["eta"].max()) if len(after["eta"]) else None}
        except binding.NepError as e:
            polish = {"unavailable": str(e)}

    # left eigenvectors of the returned pairs (Sec. 2 Eq. (nep-left)) and the resolvent's pole part
    # (Sec. 2 Eq. (resolvent)) applied to the probe block at points inside the region: one assembly
    # + band LU at the P eigenvalues, then conjugate-transpose band solves (one per step and pair)
    left_line = None
    if not args.no_polish:
        try:
            res_l = plan.result()
            P = int(len(res_l["lam"]))
            if P > 0:
                Yd = torch.zeros(2 * p.n * P, dtype=torch.float64, device="cuda")
                etad = torch.zeros(P, dtype=torch.float64, device="cuda")
                l0, l1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                l0.record()
                nc, lsteps = plan.left(Yd, etad, P, tol=1e-13, max_it=6, stream=stream)
                l1.record()
                torch.cuda.synchronize()
                c = complex(p.region["center"])
                zs = c + 0.5 * float(p.region["a"]) * np.exp(2j * np.pi * (np.arange(8) + 0.5) / 8)
                lamd = torch.from_numpy(np.ascontiguousarray(res_l["lam"]).view(np.float64).copy()).cuda()
                Xd = torch.from_numpy(np.asfortranarray(res_l["X"]).ravel(order="F").view(np.float64).copy()).cuda()
                zd = torch.from_numpy(zs.view(np.float64).copy()).cuda()
                out = torch.zeros(2 * p.n * len(zs) * p.L, dtype=torch.float64, device="cuda")
                for _ in range(3):
                    binding.apply_resolvent(p.n, P, lamd, Xd, Yd, len(zs), zd, p.L, Vd, out, stream)
                r0, r1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                r0.record()
                binding.apply_resolvent(p.n, P, lamd, Xd, Yd, len(zs), zd, p.L, Vd, out, stream)
                r1.record()
                torch.cuda.synchronize()
                eta_l = etad.cpu().numpy()
                left_line = {"pairs": int(nc), "steps": int(lsteps), "ms": l0.elapsed_time(l1),
                             "max_eta_left": float(eta_l.max()),
                             "resolvent": {"points": len(zs), "vectors": p.L, "ms": r0.elapsed_time(r1)}}
        except binding.NepError as e:
            left_line = {"unavailable": str(e)}

    # NLEIGS, static variant (Sec. 4.5) on the same problem and region: interpolation degree, one
    # FP64 band LU of R_d(sigma), then one band solve and two Gram-Schmidt passes per Arnoldi step
    nleigs_line = None
    if not args.no_nleigs:
        try:
            res_c = plan.result()
            kry = 100
            binding.nleigs_solve(split, p.region, krylov=kry, stream=stream)  # warm-up
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rn = binding.nleigs_solve(split, p.region, krylov=kry, stream=stream)
            torch.cuda.synchronize()
            ms_n = 1e3 * (time.perf_counter() - t0)
            matched = 0
            for lam in rn["lam"]:
                if len(res_c["lam"]) and np.abs(res_c["lam"] - lam).min() <= 1e-8 * max(1.0, abs(lam)):
                    matched += 1
            nleigs_line = {"degree": rn["degree"], "krylov": kry, "ms": ms_n, "pairs": int(len(rn["lam"])),
                           "max_eta": float(rn["eta"].max()) if len(rn["eta"]) else None,
                           "pairs_matching_contour": matched, "contour_pairs": int(len(res_c["lam"])),
                           "mode": "complex64 Arnoldi solves, residual inverse iteration on the converged "
                                   "Ritz pairs (FP64 residuals); compact (TOAR) basis",
                           "timing": "host clock around the synchronous call"}
            # Krylov-Schur restarts with locking: cycles of 40 steps restarted to 20 vectors
            ks_kw = dict(krylov=40, keep=20, max_restarts=30)
            binding.nleigs_solve(split, p.region, stream=stream, **ks_kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            rr = binding.nleigs_solve(split, p.region, stream=stream, **ks_kw)
            torch.cuda.synchronize()
            ms_r = 1e3 * (time.perf_counter() - t0)
            matched_r = sum(1 for lam in rr["lam"] if len(res_c["lam"]) and
                            np.abs(res_c["lam"] - lam).min() <= 1e-8 * max(1.0, abs(lam)))
            nleigs_line["restarted"] = {**ks_kw, "ms": ms_r, "pairs": int(len(rr["lam"])),
                                        "pairs_matching_contour": matched_r,
                                        "restarts": rr["info"]["restarts"],
                                        "krylov_steps": rr["info"]["krylov_steps"],
                                        "max_eta": float(rr["eta"].max()) if len(rr["eta"]) else None}
        except binding.NepError as e:
            nleigs_line = {"unavailable": str(e)}

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        csr_bytes = sum(8 * (A.shape[0] + 1) + 12 * A.nnz for A in p.mats)
        v_bytes = 16 * p.n * p.L
        # through the request server with S workers: per step the operator is uploaded
        # (nep_create_split), the request submitted with its host probe block, and its result
        # (eigenvalues, vectors, residuals) read back to the host
        Ke = max(S, args.steps)
        srv = binding.Server(workers=S)
        warm = [binding.Split.from_problem(p) for _ in range(S)]
        for t_ in [srv.submit(sp_, p.region, p.N, p.L, p.M, V=V, precision=prec) for sp_ in warm]:
            srv.wait(t_)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sps, tickets = [], []
        for _ in range(Ke):
            sps.append(binding.Split.from_problem(p))
            tickets.append(srv.submit(sps[-1], p.region, p.N, p.L, p.M, V=V, precision=prec))
        outs = [srv.wait(t_) for t_ in tickets]
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        srv.close()
        for sp_ in sps + warm:
            sp_.close()
        out_bytes = 16 * len(outs[-1]["lam"]) * (p.n + 1) + 8 * len(outs[-1]["eta"])
        # one call at a time through nep_ciss_solve (the latency a single caller sees)
        tt = []
        for it in range(3):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            sp = binding.Split.from_problem(p)
            binding.ciss_solve(sp, p.region, p.N, p.L, p.M, V=V, precision=prec)
            sp.close()
            torch.cuda.synchronize()
            if it > 0:
                tt.append(time.perf_counter() - t1)
        e2e = {"value": Ke * p.N / dt, "unit": UNIT, "h2d_bytes_per_step": csr_bytes + v_bytes,
               "d2h_bytes_per_step": out_bytes,
               "api": f"nep_server with {S} workers: nep_create_split + nep_submit (host V) + nep_server_wait, "
                      f"{Ke} requests",
               "single_call": {"value": p.N / (sum(tt) / len(tt)), "api": "nep_create_split + nep_ciss_solve"}}

    # the plain FP64 GPU path on the same workload (the metric's comparison arm), same concurrency
    fp64_arm = None
    if not args.no_fp64 and prec == binding.NEP_PREC_MIXED:
        fp64_arm = arm_bench(binding, p, binding.NEP_PREC_FP64, V, S, args.steps, args.warmup)
        fp64_arm["dtype"] = "f64"
    # the wide-band workloads (bandwidth 128 and 576), where the LU runs on the tensor core
    wide = {}
    if not args.no_wide and prec == binding.NEP_PREC_MIXED:
        for key, name, steps_w in (("c3", "drude2d_s128", 8), ("c4", "sqrt3d_s24", 4)):
            wide[key] = wide_config_bench(binding, name, measured_peaks(), 4, steps_w, rank)

    line = None
    if rank == 0:
        peaks = measured_peaks()
        cs = clk.summary()
        sm_mhz = cs["sm_mhz"] or peaks.get("sm_max_mhz", 2070.0)
        mixed = prec == binding.NEP_PREC_MIXED
        esz = 8 if mixed else 16
        alu_peak = fp32_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0)) if mixed else \
            fp64_alu_peak_tflops(peaks.get("sm_max_mhz", 2070.0))
        alu_src = ("derived: 152 SMs x 128 FP32 lanes x 2 flop x 2070 MHz" if mixed else
                   "derived: 152 SMs x 1.75 FP64 FMA/clk (measured) x 2 flop x 2070 MHz")
        s_flops = solve_flops(p.n, split.kl, split.ku, p.L, p.N)
        s_bytes = solve_bytes(p.n, split.ldab, p.L, p.N, esz)
        hbm = peaks.get("hbm_gbs", 6800.0)
        lu = float(np.mean(lu_ms))
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "single_stream": {"ms_per_step": ms_single, "value": world * p.N / (ms_single * 1e-3)},
            "vs_baseline": None, "dtype": "c64+f64" if mixed else "f64",
            "data": "synthetic",
            "config": workload_config(args.workload + (f" with N={p.N}" if args.points > 0 else ""), p),
            "execution": {"precision": args.precision,
                          "band_mb_per_step": round(p.N * p.n * split.ldab * esz / 1e6),
                          "streams": S, "concurrency": f"{S} independent plans on {S} non-blocking streams, one "
                          "host thread each; every step a full pass of its own"},
            "roofline": {"kernel": ("band_sweep_kernel x2" if split.kl + 1 <= 288 and split.kl + split.ku + 1 <= 288
                                    else ("band_solve_blocked_kernel" if mixed else "band_solve_kernel")) +
                                   " (forward + backward banded substitution, "
                                   f"{p.N} points x {p.L} right-hand sides in one launch)",
                         "bound": "hbm", "achieved": s_bytes / (solve_ms * 1e-3) / 1e9, "peak": hbm,
                         "unit": "GB/s", "frac": s_bytes / (solve_ms * 1e-3) / 1e9 / hbm,
                         "traffic": SOLVE_TRAFFIC.get((args.workload, args.precision)),
                         "ms_per_launch": solve_ms,
                         "peak_source": "measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs)",
                         "algorithmic_bytes": s_bytes,
                         "alu": {"achieved_tflops": s_flops / (solve_ms * 1e-3) / 1e12, "peak_tflops": alu_peak,
                                 "frac": s_flops / (solve_ms * 1e-3) / 1e12 / alu_peak, "peak_source": alu_src,
                                 "flops": s_flops}},
            "factor": {"kernel": "lu_col_kernel" if split.kl <= 64 and split.kl + split.ku <= 128 else
                       ("lu_tc_kernel" if mixed else "lu_wide_kernel"),
                       "ms": lu, "achieved_tflops": lu_flops(p.n, split.kl, split.ku, p.N) / (lu * 1e-3) / 1e12,
                       "peak_tflops": alu_peak,
                       "frac": lu_flops(p.n, split.kl, split.ku, p.N) / (lu * 1e-3) / 1e12 / alu_peak},
            "stages_ms": stage, "clocks": cs, "gpu_launches": int(launches),
            "gpu_launches_per_step": int(launches) // max(1, args.steps),
            "result": {"nconv": int(len(res["lam"])), "hankel_rank": res["m"], "max_eta": float(res["eta"].max())
                       if len(res["eta"]) else None, "max_backward": res["info"]["max_backward"],
                       "max_sweeps": res["info"]["max_sweeps"], "svd_sweeps": res["info"]["svd_sweeps"],
                       "flags": res["flags"]},
        }
        if e2e:
            line["e2e"] = e2e
        if symmetric:
            line["symmetric"] = symmetric
        if polish:
            line["polish"] = polish
        if left_line:
            line["left"] = left_line
        if nleigs_line:
            line["nleigs"] = nleigs_line
        if fp64_arm:
            line["fp64"] = fp64_arm
            line["mixed_over_fp64"] = value / (world * fp64_arm["value"])
        for key, blk in wide.items():
            line[key] = blk
        if not args.no_serving:
            line["serving"] = serving_bench(binding, prec, args.serving_requests, 0, 4, args.serving_smax)
            # the same stream with shared launches: two workers, batches of up to four requests
            line["serving_batched"] = serving_bench(binding, prec, args.serving_requests, 0, 2, args.serving_smax,
                                                    max_batch=4, fp64=False)
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(p)
            cores = max(1, min(32, os.cpu_count() or 1))
            if "c3" in wide:
                p3 = synth.config_problem("drude2d_s128", seed=0)
                v3 = cpu_sample_points(p3, 2 * cores, cores)
                line["c3"]["cpu_baseline"] = {"value": v3, "unit": UNIT, "cores": cores, "kind": "oracle",
                                              "sample": f"quadrature solves at {2 * cores} of the 128 nodes of "
                                                        "drude2d_s128 (assembly, band LU, FP64 refinement), "
                                                        f"{cores} threads over points",
                                              "one_thread": {"value": cpu_sample_points(p3, 1, 1), "unit": UNIT,
                                                             "sample": "the solve at 1 node, one thread"}}
            if "c4" in wide:
                # one node per thread: about 70 GF of band LU per node, tens of seconds each
                p4 = synth.config_problem("sqrt3d_s24", seed=0)
                v4 = cpu_sample_points(p4, cores, cores)
                line["c4"]["cpu_baseline"] = {"value": v4, "unit": UNIT, "cores": cores, "kind": "oracle",
                                              "sample": f"quadrature solves at {cores} of the 64 nodes of "
                                                        "sqrt3d_s24 (assembly, band LU, FP64 refinement), one node "
                                                        f"on each of {cores} threads",
                                              "seconds_per_node_one_thread": cores / v4}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
