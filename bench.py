"""Benchmark: amplitudes/s and histories/s of the reduced-history path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload NAME] [--impl ours|reference]

A step is one evaluation of every job of the workload's batch: counter
reset, prefix expansion (checkpoint table), persistent history kernel,
fixed-order reduction.  Inputs (programs, bit strings) are resident in HBM
when the timed region starts; the L2 is flushed (a 512 MiB write) between
timed steps.  Rank 0 prints one JSON line.
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
sys.path.insert(0, ROOT)

METRIC = "amplitudes/s and histories/s on 1 B300, batched+learned vs plain, fidelity≥0.999"

def workload_jobs(name, rank=0, outputs=None):
    from workloads import qaoa_workload, qw_workload
    if name == "qw100":
        n_out = outputs or 4096
        w = qw_workload(n_out=n_out, seed=0x5EED0005 + rank)
        return [w], {"workload": f"qw100_t16_{n_out}out_exact", "qubits": 100, "steps": 16,
                     "outputs": n_out, "input_support": 2, "eps": 0.0}
    if name == "qw100+qaoa":
        ws = [qw_workload(seed=0x5EED0005 + rank)]
        for n in (16, 20, 24):
            ws.append(qaoa_workload(n, 2, n_out=1024, eps=1e-4, seed=0x5EED0003 + rank))
        return ws, {"workload": "qw100_t16_4096out_exact+qaoa16_20_24_p2_1024out_eps1e-4",
                    "outputs": 4096 + 3 * 1024}
    raise SystemExit(f"unknown workload {name}")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[3 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(self.rows)}


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


# ------------------------------------------------------------------ CPU oracle timing

def oracle_sample(jobs, budget_s=15.0, max_outputs=None):
    """Times the C oracle (Algorithm 2 at its own autotuned cuts, all host
    threads) on a bounded sample of each job's outputs; returns rates."""
    from oracle import feynman
    threads = os.cpu_count() or 1
    tot_out = 0
    tot_hist = 0
    tot_time = 0.0
    desc = []
    per_job_budget = budget_s / len(jobs)
    for w in jobs:
        c1, c2, _ = feynman.autotune(w.circuit)
        k = max(1, threads)
        t_used = 0.0
        done = 0
        hist = 0
        while t_used < per_job_budget and done < len(w.outputs):
            outs = w.outputs[done:done + k]
            t0 = time.perf_counter()
            _, cnt = feynman.run(w.circuit, w.inputs, outs, eps=w.eps, c1=c1, c2=c2, threads=threads)
            dt = time.perf_counter() - t0
            t_used += dt
            done += len(outs)
            hist += int(cnt["completed"].sum())
            if max_outputs and done >= max_outputs:
                break
        tot_out += done
        tot_hist += hist
        tot_time += t_used
        desc.append(f"{w.name}: {done} of {len(w.outputs)} outputs")
    return {"amplitudes_per_s": tot_out / tot_time, "histories_per_s": tot_hist / tot_time,
            "seconds": tot_time, "cores": threads, "sample": "; ".join(desc)}


def run_reference(args):
    rank, world, local = dist_setup(args)
    if rank != 0:
        return
    jobs, cfg = workload_jobs(args.workload, 0, args.outputs)
    for _ in range(args.warmup):
        oracle_sample(jobs, budget_s=2.0, max_outputs=1)
    rates = []
    samp = None
    for _ in range(args.steps):
        samp = oracle_sample(jobs, budget_s=max(5.0, 60.0 / max(args.steps, 1)))
        rates.append(samp["amplitudes_per_s"])
    v = statistics.mean(rates)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "amplitudes/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * samp["seconds"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded circuits and requests)",
            "config": cfg, "histories_per_s": samp["histories_per_s"],
            "cpu_baseline": {"value": v, "unit": "amplitudes/s", "cores": samp["cores"],
                             "kind": "oracle", "sample": samp["sample"]},
            "e2e": {"value": v, "unit": "amplitudes/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arm

def run_ours(args):
    import torch
    import paper_2608_01467_b300 as fs
    rank, world, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    jobs, cfg = workload_jobs(args.workload, rank, args.outputs)
    b = fs.Batch(engine=args.engine)
    circs = []
    for w in jobs:
        C = fs.Circuit(w.circuit)
        C.set_input(w.inputs)
        circs.append(C)
        b.add(C, w.outputs, w.eps)
    ws_bytes = b.plan()
    b.allocate(dev)
    stream = torch.cuda.current_stream(dev)
    b.upload(stream)
    engine, compile_ms = b.engine()
    b.time_kernels(True)
    n_out = b.total_outputs
    flush = torch.empty(512 << 20, dtype=torch.uint8, device=dev)

    for _ in range(max(args.warmup, 3)):
        b.run(stream)
        b.finish(stream)
    stats0 = b.finish(stream)

    # timed region: device time of each step with CUDA events on the launch stream
    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    barrier(world)
    torch.cuda.synchronize(dev)
    step_ms, hist_ms, pre_ms, red_ms = [], [], [], []
    completed = 0
    for _ in range(args.steps):
        flush.zero_()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        b.run(stream)
        e1.record(stream)
        st = b.finish(stream)
        step_ms.append(e0.elapsed_time(e1))
        p, h, r = b.kernel_ms()
        pre_ms.append(p)
        hist_ms.append(h)
        red_ms.append(r)
        completed += sum(s["completed"] for s in st)
    torch.cuda.synchronize(dev)
    barrier(world)
    clocks = sampler.stop()
    t_total = sum(step_ms) / 1000.0
    t_max = max_over_ranks(t_total, world, dev)
    outs_all = sum_over_ranks(n_out * args.steps, world, dev)
    hist_all = sum_over_ranks(completed, world, dev)
    value = outs_all / t_max
    hist_rate = hist_all / t_max

    # end to end through the public API with host buffers: H2D of the step's
    # programs and bit strings, run, D2H of the amplitudes, every step
    host_amp = torch.empty(b.amp.shape, dtype=b.amp.dtype, pin_memory=True)
    barrier(world)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        b.upload(stream)
        b.run(stream)
        host_amp.copy_(b.amp, non_blocking=True)
        b.finish(stream)
    torch.cuda.synchronize(dev)
    t_e2e = max_over_ranks(time.perf_counter() - t0, world, dev)
    e2e = sum_over_ranks(n_out * args.steps, world, dev) / t_e2e

    # roofline of the history kernel (the dominant kernel): algorithmic
    # integer ops and FP64 instructions of the root + suffix per launch, from
    # the library's per-region work of each job times the region executions
    peaks = fs.api.probe_peaks()
    int_ops = 0.0
    fp_ops = 0.0
    for ji, w in enumerate(jobs):
        iw, fw = b.region_work(ji)
        s0 = stats0[ji]
        pairs = len(w.outputs) * len(w.inputs)
        root_runs = s0["table_entries"] << s0["A_r"]          # live checkpoints x 2^A_r
        suffix_runs = s0["completed"] if w.eps > 0 else pairs << (s0["A_p"] + s0["A_r"] + s0["A_s"])
        int_ops += iw[1] * root_runs + iw[2] * suffix_runs + iw[3] * s0["completed"]
        fp_ops += fw[1] * root_runs + fw[2] * suffix_runs + fw[3] * s0["valid"]
    h_s = statistics.mean(hist_ms) / 1000.0
    sm_max = clocks["sm_max_mhz"] or 2032.0
    int_peak = peaks["sms"] * 128 * sm_max * 1e6
    int_frac = int_ops / h_s / int_peak
    fp_frac = fp_ops / h_s / peaks["dfma_per_s"]
    if int_frac >= fp_frac:
        roof = {"bound": "alu", "achieved": int_ops / h_s / 1e9, "peak": int_peak / 1e9,
                "unit": "Gop/s", "frac": int_frac}
    else:
        roof = {"bound": "alu", "achieved": fp_ops / h_s / 1e9, "peak": peaks["dfma_per_s"] / 1e9,
                "unit": "GFP64-inst/s", "frac": fp_frac}
    roof.update({"traffic": None, "kernel": "history_kernel",
                 "history_kernel_ms": statistics.mean(hist_ms),
                 "prefix_kernel_ms": statistics.mean(pre_ms), "reduce_kernel_ms": statistics.mean(red_ms),
                 "int_ops_per_launch": int_ops, "fp64_inst_per_launch": fp_ops,
                 "int_frac": int_frac, "fp64_frac": fp_frac,
                 "int_peak_note": "derived: SMs x 128 lanes x max SM clock",
                 "fp64_peak_measured_dfma_per_s": peaks["dfma_per_s"],
                 "int_peak_measured_ops_per_s": peaks["int_ops_per_s"]})

    line = {"metric": METRIC, "value": value, "unit": "amplitudes/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * t_max / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic (seeded circuits and requests)",
            "config": dict(cfg, l2="flushed between steps (512 MiB write)",
                           parallelism=f"outputs sharded, {world} replica(s)",
                           workspace_bytes=ws_bytes, engine=engine,
                           engine_compile_ms=round(compile_ms, 1)),
            "histories_per_s": hist_rate, "clocks": clocks,
            "e2e": {"value": e2e, "unit": "amplitudes/s",
                    "h2d_bytes_per_step": int(b.static_bytes()),
                    "d2h_bytes_per_step": int(16 * n_out)},
            "gpu_launches": b.launch_count() * args.steps,
            "roofline": roof}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        samp = oracle_sample(jobs, budget_s=args.cpu_seconds)
        line["cpu_baseline"] = {"value": samp["amplitudes_per_s"], "unit": "amplitudes/s",
                                "cores": samp["cores"], "kind": "oracle", "sample": samp["sample"],
                                "histories_per_s": samp["histories_per_s"]}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="qw100")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--outputs", type=int, default=None, help="requested outputs (small profiling cases)")
    ap.add_argument("--engine", default="straight", choices=["straight", "interp"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
