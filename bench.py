"""Benchmark: digital adiabatic state-vector evolution of Z2 lattice gauge
theory on GB300 (one JSON line on stdout).

Workload (default): 2+1D Z2 LGT on the 4x4 periodic lattice, 32 link qubits,
complex64 state (34.4 GB, in place, far larger than L2), H(s) = -sum sigma^x
- s*lambda*sum_p U_p with lambda = 3, T = 20, M = 500 symmetric Trotter steps
from |+>^32.  One benchmark step = one whole adiabatic run through the C ABI:
|+> initialisation, the M Trotter steps, and the observables (<H>, <U_p>, 2x2
Wilson loop, Gauss-law stars, sigma^z/sigma^x, W/V loops, fidelity against a
device-resident reference state).  Metric: Trotter steps per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload 4x4|4x3|2x2x2] [--decomp sym|first]

Multi-GPU: replicas only (the runs are independent); one process per GPU
under torchrun, max-over-ranks time, value = all ranks' Trotter steps / time.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {
    "4x4": dict(d=2, L=(4, 4), lam=3.0, T=20.0, M=500,
                name="2+1D Z2 LGT 4x4 periodic, 32 link qubits, complex64 (34.4 GB), lambda=3, T=20, M=500"),
    "4x3": dict(d=2, L=(4, 3), lam=3.0, T=20.0, M=500,
                name="2+1D Z2 LGT 4x3 periodic, 24 link qubits, complex64, lambda=3, T=20, M=500"),
    "2x2x2": dict(d=3, L=(2, 2, 2), lam=1.0, T=15.0, M=300,
                  name="3+1D Z2 LGT 2x2x2 periodic, 24 link qubits, complex64, lambda=1, T=15, M=300"),
    # small case of the 32-qubit kernel for profiler captures (2.1 GB state)
    "7x2": dict(d=2, L=(7, 2), lam=3.0, T=2.0, M=20,
                name="2+1D Z2 LGT 7x2 periodic, 28 link qubits, complex64 (2.1 GB), lambda=3, T=2, M=20"),
}
METRIC = "Trotter steps/s"


def dist_info():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.p = None

    def stop(self):
        if not self.p:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        out, _ = self.p.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                smax.append(float(f[1]))
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def aggregate(elapsed_s, trotter_steps_per_rank, dist=None, device=None):
    """Whole-job throughput of independent replicas: every rank's Trotter
    steps over the slowest rank's time (max over ranks, no data exchange)."""
    world = 1
    if dist is not None and dist.is_initialized():
        import torch
        world = dist.get_world_size()
        t = torch.tensor([float(elapsed_s)], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        elapsed_s = float(t.item())
    return elapsed_s, trotter_steps_per_rank * world / elapsed_s


def measured_peak():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def kernel_name(variant, info):
    """The pass kernel a plan runs (see z2_ctx_set_option / z2_autotune)."""
    ring_ok = info.n_groups > 1 and 10 <= info.tile_bits <= 13
    if variant == 4 and info.n_groups > 1 and 12 <= info.tile_bits <= 13:
        return f"pass_kernel_ring<{info.tile_bits},5,RX>"
    if variant in (0, 5) and info.n_groups > 1 and 12 <= info.tile_bits <= 13:
        return f"pass_kernel_ring<{info.low_tile_bits},4,RX>+<{info.tile_bits},5,RX>"
    if variant in (0, 3) and ring_ok:
        if info.low_tile_bits != info.tile_bits:  # low group on the smaller tile
            return f"pass_kernel_ring<{info.low_tile_bits},4,RX>+<{info.tile_bits},4,RX>"
        return f"pass_kernel_ring<{info.tile_bits},4,RX>"
    if variant == 2:
        return f"pass_kernel_tma<float2,{info.tile_bits},RX>"
    return f"pass_kernel_packed<{info.tile_bits},4,RX>"


def l2_note(state_bytes):
    """How the timed region relates to the 129 MB L2 (inputs are not flushed
    between timed steps; the state is the input every pass streams)."""
    if state_bytes > 4 * 129e6:
        return "state (%.1f GB) >> L2 (129 MB): no flush needed" % (state_bytes / 1e9)
    return ("state (%.0f MB) about the size of L2 (129 MB), no flush: every pass streams the whole state, "
            "part of it from L2" % (state_bytes / 1e6))


def recorded_traffic(n, kernel):
    """DRAM bytes per pass launch of `kernel` from the committed ncu record,
    scaled to n qubits; None if the record is missing, names another kernel,
    or the kernel source changed since."""
    import hashlib
    try:
        rec = {}
        for line in open(os.path.join(ROOT, "profiles", "pass_kernel_ring_traffic.txt")):
            if line.strip() and not line.startswith("#"):
                k, v = line.split(None, 1)
                rec[k] = v.strip()
        if rec["kernel"] != kernel:
            return None
        src = open(os.path.join(ROOT, rec["source"]), "rb").read()
        if hashlib.sha256(src).hexdigest() != rec["source_sha256"]:
            return None
        return float(rec["dram_bytes_per_launch"]) * 2.0 ** (n - int(rec["qubits"]))
    except Exception:
        return None


_CPU_STATE = {}


def cpu_model():
    """The host CPU's model name (lscpu), else the machine type."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=20).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def cpu_baseline(wl, decomp, budget_s=12.0):
    """The FP64 oracle (plain C, OpenMP over all host cores) timed on a real
    state: Trotter steps of the workload's own lattice when it has at most 30
    links, else of the 5x3 periodic lattice (30 qubits, a 17.2 GB FP64
    state), with the workload's lambda and dt; at least one step and as many
    as the budget allows (the state is allocated once per process).  A
    30-qubit rate is extrapolated to the workload by the 2^N * N work ratio
    of a Trotter step (x4.27 for 32 qubits), and the sample says so."""
    import numpy as np

    import oracle
    from oracle.lattice import Lattice as OLattice

    n_w = wl["d"] * int(np.prod(wl["L"]))
    d, L = (wl["d"], tuple(wl["L"])) if n_w <= 30 else (2, (5, 3))
    ol = OLattice(d, L)
    n = ol.n_links
    key = (d, L)
    if key not in _CPU_STATE:
        _CPU_STATE.clear()
        _CPU_STATE[key] = oracle.init_plus(n)
    psi = _CPU_STATE[key]
    masks = ol.plaq_masks()
    steps = 0
    t0 = time.perf_counter()
    while steps < 1 or (time.perf_counter() - t0 < budget_s and steps < wl["M"]):
        oracle.evolve(psi, masks, wl["lam"], wl["T"], wl["M"], decomp, 0, steps, steps + 1)
        steps += 1
    el = time.perf_counter() - t0
    rate = steps / el
    scale = ((1 << n) * n) / ((1 << n_w) * n_w)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    where = f"{'x'.join(map(str, L))} lattice ({n} qubits, FP64 state {16 * 2 ** n / 1e9:.1f} GB)"
    sample = (f"{steps} {'symmetric' if decomp else 'first-order'} Trotter steps of the {where} in {el:.1f} s "
              f"= {rate:.4f} steps/s on {cores} cores of {cpu_model()}")
    if n != n_w:
        sample += f", extrapolated to {n_w} qubits by the 2^N*N work ratio (x{1 / scale:.3f})"
    return {"value": rate * scale, "unit": METRIC, "cores": cores, "kind": "oracle", "cpu": cpu_model(),
            "sample": sample}


def run_reference(args, wl, decomp):
    rank, world, _ = dist_info()
    if rank != 0:
        return
    # W warm-up + K timed steps, each a bounded sample of the oracle (at least
    # one Trotter step on the real state)
    budget = max(2.0, 60.0 / max(1, args.steps + args.warmup))
    for _ in range(args.warmup):
        cpu_baseline(wl, decomp, budget_s=0.0)
    vals = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        vals.append(cpu_baseline(wl, decomp, budget_s=budget))
    el = time.perf_counter() - t0
    v = statistics.median(x["value"] for x in vals)
    cb = dict(vals[0])
    cb["value"] = v
    line = {"metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * el / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl["name"], "decomp": "symmetric" if decomp else "first-order"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0,
                                        "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def run_sweep(args):
    """Batched lambda sweep: 256 seeded runs (3x3 / 4x3 / 2x2x2 lattices,
    lambda ~ U[0,6), T ~ U[5,20], M ~ U{100..400}, symmetric, complex64) in
    each sweep mode; runs/s per mode, plans rebuilt inside every timed call."""
    import torch

    import paper_1910_08020_gb300 as z2
    from paper_1910_08020_gb300 import workloads

    torch.cuda.set_device(0)
    ctx = z2.Context(0)
    if args.variant:
        z2.z2_ctx_set_option(ctx.handle, z2.Z2_OPT_PASS_VARIANT, args.variant)
    if getattr(args, "split_low", 0):
        z2.z2_ctx_set_option(ctx.handle, z2.Z2_OPT_SPLIT_LOW_BITS, args.split_low)
    specs = workloads.sweep_specs(args.sweep_runs)
    arr = z2.run_specs(specs)
    steps = sum(sp["M"] for sp in specs)
    warm = z2.run_specs(workloads.sweep_specs(6, seed=1))
    for mode in (0, 1, 2, 3):
        z2.z2_sweep(ctx.handle, warm, mode=mode, n_streams=args.streams)
    out = {}
    for name, mode in (("plain", 0), ("streams", 1), ("graphs", 2), ("persistent", 3)):
        z2.z2_ctx_flush_plans(ctx.handle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        res = z2.z2_sweep(ctx.handle, arr, mode=mode, n_streams=args.streams)
        el = time.perf_counter() - t0
        assert all(r.status == 0 for r in res)
        out[name] = {"runs_per_s": len(specs) / el, "seconds": el, "trotter_steps_per_s": steps / el}
    best = max(("streams", "graphs", "persistent"), key=lambda k: out[k]["runs_per_s"])
    line = {"metric": "lambda-sweep runs/s", "value": out[best]["runs_per_s"], "unit": "runs/s", "n_gpus": 1,
            "best_mode": best,
            "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"{len(specs)} adiabatic runs, lattices 3x3 (18q) / 4x3 (24q) / 2x2x2 (24q), "
                                   "lambda~U[0,6), T~U[5,20], M~U{100..400}, symmetric, complex64, seed 20191018",
                       "streams": args.streams, "total_trotter_steps": steps},
            "modes": out, "speedup_vs_plain": {k: out[k]["runs_per_s"] / out["plain"]["runs_per_s"] for k in out}}
    print(json.dumps(line), flush=True)
    ctx.close()


def run_serve(args):
    """Serving: a seeded Poisson request stream (lattices 2x2 .. 5x3 and
    2x2x2, lambda ~ U[0,6], M ~ U{50..500}, T = 0.04 M, symmetric) submitted
    on its own clock to the continuous-batching server, then the same stream
    through the plain FIFO path (one run at a time, in arrival order)."""
    import numpy as np
    import torch

    import paper_1910_08020_gb300 as z2
    from paper_1910_08020_gb300 import workloads

    torch.cuda.set_device(0)
    ctx = z2.Context(0)
    lats = [l for l in workloads.SERVE_LATTICES if l[0] * int(np.prod(l[1])) <= args.serve_max_qubits]
    reqs = workloads.poisson_stream(args.serve_count, rate=args.serve_rate, lattices=lats)
    gpu_s_offered = None

    def pct(v, q):
        return float(np.percentile(np.array(v), q))

    # warm-up: one request per lattice through both paths
    for d, L in lats:
        lat = z2.Lattice(d, L)
        g = torch.empty(1 << lat.n_links, dtype=torch.complex64, device="cuda")
        z2.z2_run(ctx.handle, lat.handle, z2.params(1.0, 2.0, 50), g)
        del g
    torch.cuda.synchronize()

    srv = z2.z2_server_create(ctx.handle, hbm_budget=0, max_slots=args.serve_slots)
    t0 = time.monotonic()
    tickets = []
    for rq in reqs:
        delay = rq["arrival"] - (time.monotonic() - t0)
        if delay > 0:
            time.sleep(delay)
        tickets.append(z2.z2_server_submit(srv, rq))
    lat_s = []
    for tk in tickets:
        rc, res = z2.z2_server_wait(srv, tk, timeout_s=3600)
        assert rc == 0
        q, r = z2.z2_server_request_times(srv, tk)
        lat_s.append(q + r)
    t_end = time.monotonic() - t0
    st = z2.z2_server_stats(srv)
    z2.z2_server_destroy(srv)
    served = {"p50_s": pct(lat_s, 50), "p99_s": pct(lat_s, 99), "runs_per_s": len(reqs) / t_end,
              "hbm_peak_gb": st.hbm_peak / 1e9, "slots": args.serve_slots}

    # the plain FIFO path: one run at a time in arrival order
    t0 = time.monotonic()
    fifo = []
    run_time = 0.0
    for rq in reqs:
        delay = rq["arrival"] - (time.monotonic() - t0)
        if delay > 0:
            time.sleep(delay)
        lat = z2.Lattice(rq["d"], rq["L"])
        g = torch.empty(1 << lat.n_links, dtype=torch.complex64, device="cuda")
        ts = time.monotonic()
        z2.z2_run(ctx.handle, lat.handle, z2.params(rq["lam"], rq["T"], rq["M"]), g)
        run_time += time.monotonic() - ts
        fifo.append(time.monotonic() - t0 - rq["arrival"])
        del g
    t_fifo = time.monotonic() - t0
    plain = {"p50_s": pct(fifo, 50), "p99_s": pct(fifo, 99), "runs_per_s": len(reqs) / t_fifo}
    offered = run_time / reqs[-1]["arrival"]
    line = {"metric": "serving p50/p99 latency and runs/s", "value": served["runs_per_s"], "unit": "runs/s",
            "n_gpus": 1, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"{len(reqs)} Poisson requests at {args.serve_rate}/s, lattices "
                                   + ", ".join("x".join(map(str, L)) for _, L in lats)
                                   + ", lambda~U[0,6], M~U{50..500}, T=0.04M, symmetric, complex64",
                       "offered_gpu_seconds_per_second": offered},
            "served": served, "plain_fifo": plain,
            "speedup_runs_per_s": served["runs_per_s"] / plain["runs_per_s"]}
    print(json.dumps(line), flush=True)
    ctx.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="4x4", choices=sorted(WORKLOADS))
    ap.add_argument("--decomp", default="sym", choices=["sym", "first"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--variant", type=int, default=0, help="pass kernel: 0 auto, 1 direct (packed), 2 TMA, 3 ring, 4 ring with 32 pairs per thread, "
                    "5 ring with 32 pairs per thread on the strided groups")
    ap.add_argument("--tile-bits", type=int, default=0)
    ap.add_argument("--split-low", type=int, default=0,
                    help="ring plans with two strided groups: bits of the split group at the bottom (0 = automatic)")
    ap.add_argument("--autotune", action="store_true",
                    help="time every tile size x kernel variant before the warm-up and run the fastest "
                         "(default: the automatic plan)")
    ap.add_argument("--no-autotune", action="store_true", help="(default) run the automatic plan")
    ap.add_argument("--mode", default="run", choices=["run", "sweep", "serve"],
                    help="run: the headline workload; sweep: batched lambda sweep; serve: request stream")
    ap.add_argument("--sweep-runs", type=int, default=256)
    ap.add_argument("--streams", type=int, default=8)
    ap.add_argument("--serve-count", type=int, default=2000)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-max-qubits", type=int, default=30)
    ap.add_argument("--serve-slots", type=int, default=16)
    args = ap.parse_args()
    wl = WORKLOADS[args.workload]
    decomp = 1 if args.decomp == "sym" else 0
    if args.impl == "reference":
        run_reference(args, wl, decomp)
        return
    if args.mode == "sweep":
        run_sweep(args)
        return
    if args.mode == "serve":
        run_serve(args)
        return

    import numpy as np
    import torch

    import paper_1910_08020_gb300 as z2

    rank, world, local = dist_info()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist_mod
        dist_mod.init_process_group("nccl")
        dist = dist_mod
    z2.load()
    ctx = z2.Context(local)
    if args.variant:
        z2.z2_ctx_set_option(ctx.handle, z2.Z2_OPT_PASS_VARIANT, args.variant)
    if getattr(args, "split_low", 0):
        z2.z2_ctx_set_option(ctx.handle, z2.Z2_OPT_SPLIT_LOW_BITS, args.split_low)
    if args.tile_bits:
        z2.z2_ctx_set_option(ctx.handle, z2.Z2_OPT_TILE_BITS, args.tile_bits)
    lat = z2.Lattice(wl["d"], wl["L"])
    n = lat.n_links
    p = z2.params(wl["lam"], wl["T"], wl["M"], decomp, z2.Z2_C64)
    stream = torch.cuda.current_stream()
    state = torch.empty(1 << n, dtype=torch.complex64, device="cuda")
    ref = torch.empty_like(state)
    z2.z2_init_plus(ctx.handle, lat.handle, z2.Z2_C64, ref, stream)  # reference state for the fidelity
    tune = None
    if args.autotune and not args.no_autotune and not args.variant and not args.tile_bits:
        tr = z2.z2_autotune(ctx.handle, lat.handle, z2.Z2_C64, state, stream)
        tune = {"tile_bits": tr.tile_bits, "variant": tr.variant, "us_per_step": tr.us_per_step,
                "candidates": tr.n_candidates}
    info = z2.z2_evolve_plan_info(ctx.handle, lat.handle, p, 0, wl["M"])
    state_bytes = lat.state_bytes(z2.Z2_C64)

    ev_pass = []

    def step(record=False):
        z2.z2_init_plus(ctx.handle, lat.handle, z2.Z2_C64, state, stream)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        z2.z2_evolve(ctx.handle, lat.handle, p, state, 0, wl["M"], stream)
        e1.record(stream)
        res = z2.z2_measure(ctx.handle, lat.handle, p, state, 1.0, ref, stream)
        if record:
            ev_pass.append((e0, e1))
        return res

    for _ in range(args.warmup):
        res = step()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    l0 = z2.z2_ctx_launch_count(ctx.handle)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    for _ in range(args.steps):
        res = step(record=True)
    t_end.record(stream)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ck = clocks.stop()
    launches = z2.z2_ctx_launch_count(ctx.handle) - l0
    elapsed = t_start.elapsed_time(t_end) / 1000.0
    evolve_s = sum(a.elapsed_time(b) for a, b in ev_pass) / 1000.0
    elapsed, value = aggregate(elapsed, wl["M"] * args.steps, dist, device="cuda")
    pass_launches = info.n_passes * args.steps
    avg_pass = evolve_s / pass_launches
    # algorithmic unit: one Trotter step reads and writes the state once
    # (16 * 2^N bytes); one pass launch advances M / n_passes of a step
    step_bytes = 2.0 * state_bytes
    steps_per_launch = wl["M"] / info.n_passes
    alg_bytes = step_bytes * steps_per_launch
    peak, peak_kind = measured_peak()
    achieved = alg_bytes / avg_pass / 1e9
    pass_gbs = step_bytes / avg_pass / 1e9  # streaming rate of a pass (reads + writes the state once)

    # end to end through the public API: plans (phase tables, pass lists) are
    # rebuilt and uploaded from host memory every step, results read back
    e2e_t = []
    h2d = info.n_tables * 33 * 8 + info.n_passes * 40  # phase tables + 40-byte pass steps
    for _ in range(max(1, min(args.steps, 3))):  # a sample of whole runs is enough for the mean
        z2.z2_ctx_flush_plans(ctx.handle)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        z2.z2_run(ctx.handle, lat.handle, p, state, ref, stream)
        e2e_t.append(time.perf_counter() - t0)
    e2e_v = wl["M"] * world / statistics.mean(e2e_t)
    d2h = 8 * 256

    d = z2.results_dict(res, lat.info)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cb = cpu_baseline(wl, decomp)
    if rank == 0:
        kname = kernel_name(args.variant or (tune or {}).get("variant", 0), info)
        line = {
            "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c64 (fp32 arithmetic, fp64 tables/reductions)",
            "data": "synthetic",
            "config": {"workload": wl["name"], "decomp": "symmetric" if decomp else "first-order",
                       "step": "one whole adiabatic run (init, M Trotter steps, observables)",
                       "trotter_steps_per_bench_step": wl["M"], "tile_bits": info.tile_bits,
                       "low_group_tile_bits": info.low_tile_bits,
                       "qubit_groups": info.n_groups, "passes_per_run": info.n_passes,
                       "l2": l2_note(state_bytes),
                       "parallelism": f"replicas x{world}",
                       "fidelity_ref": "device-resident reference state (|+>^N)", "autotune": tune},
            "gpu_launches": launches,
            "roofline": {"bound": "hbm", "kernel": kname,
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_kind": peak_kind,
                         "traffic": recorded_traffic(n, kname),
                         "algorithmic_bytes_per_launch": alg_bytes, "avg_launch_ms": avg_pass * 1e3,
                         "unit_of_work": "one Trotter step = one read + one write of the state "
                                         f"({step_bytes / 1e9:.3f} GB); {steps_per_launch:.4f} steps per launch",
                         "per_pass": {"bytes": step_bytes, "achieved": pass_gbs, "frac": pass_gbs / peak}},
            "e2e": {"value": e2e_v, "unit": "steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "clocks": ck,
            "result": {"energy": d["energy"], "mean_plaq": d["mean_plaq"], "wilson_2x2": d["wilson_2x2"],
                       "mean_star": d["mean_star"], "norm": d["norm"], "fidelity": d["fidelity"]},
        }
        if cb:
            line["cpu_baseline"] = cb
        print(json.dumps(line), flush=True)
    ctx.close()
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
