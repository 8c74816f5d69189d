#!/usr/bin/env python3
"""Throughput benchmark of the DOCH hot path on one GB300 (or N, weak scaling).

Workload (one step): a periodic 10^4 x 10^4 lattice (n = 1e8 spins) with
+-1 nearest-neighbour couplings held as int8 (2e8 edges), FP32 iterates,
1 replica: reset x to the seeded start x0, 500 DOCH iterations
x <- cbrt(((J + alpha I) x) / beta) (Eq. FPE, Algorithm 1), then sign
rounding, the exact int64 Ising energy and cut, and the best replica.
alpha = lambda_max(-J) by the Wigner estimate (n >= 1e4), beta by Eq.
alphabeta; both set up before the timed region. Inputs are synthetic and
seeded (paper_2509_01928_gb300.inputs), larger than L2 (1.2 GB live).

Metric: spin-updates/s = n * replicas * iterations / second, whole job.
Under torchrun every rank solves its own seeded instance (no data-path
collective; "scaling": "weak"); time is the max over ranks.

--impl reference times the FP64 oracle (the plain CPU restatement of the
method, test infrastructure) on a bounded sample of the same workload on
the host cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "spin-updates/s (n*replicas*iters/s)"
UNIT = "spin-updates/s"
SEED = 2
BYTES_PER_SITE = 10  # read x (4 B) + right and down couplings (2 B) + write x (4 B)
DOMINANT = "torus_f32_r1_vec4"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "torus_f32_r1_vec4_10000x10000.md")


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def recorded_traffic():
    """Per-launch DRAM bytes of the dominant kernel from the committed ncu
    summary, if it was taken on the kernel source as it is now."""
    try:
        txt = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    m_bytes = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m_hash = re.search(r"kernel_source_sha256:\s*([0-9a-f]+)", txt)
    if not (m_bytes and m_hash):
        return None
    src = open(os.path.join(ROOT, "paper_2509_01928_gb300", "csrc", "k_torus.cu"), "rb").read()
    if hashlib.sha256(src).hexdigest() != m_hash.group(1):
        return None
    return float(m_bytes.group(1))


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id=None):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd += ["-i", self.gpu_id]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


def cpu_oracle_sample(lr: int, lc: int, iters: int):
    """Time the FP64 oracle (single thread) on an lr x lc lattice sample."""
    import oracle as O
    from paper_2509_01928_gb300 import inputs as I

    t = I.torus_pm1(lr, lc, seed=SEED)
    x0 = I.x0_uniform(t.n, 1, seed=SEED)
    P = O.Problem(t)
    alpha, beta = O.alpha_beta(t, eta=1.0, method="wigner")
    t0 = time.perf_counter()
    x = O.doch(P, x0, alpha, beta, iters)
    O.energy_int(P, O.sign(x))
    dt = time.perf_counter() - t0
    return t.n * iters, dt


def run_reference(args):
    rank, world, _ = env_rank()
    if rank != 0:
        return
    lr = lc = args.ref_size
    iters = args.ref_iters
    for _ in range(args.warmup):
        cpu_oracle_sample(lr, lc, iters)
    tot_u, tot_t = 0, 0.0
    for _ in range(args.steps):
        u, dt = cpu_oracle_sample(lr, lc, iters)
        tot_u += u
        tot_t += dt
    value = tot_u / tot_t
    sample = f"torus {lr}x{lc} int8 +-1, {iters} FP64 DOCH iterations + sign + int64 energy per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot_t / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": f"torus2d {args.size}x{args.size} +-1 int8, DOCH (oracle on a bounded sample)",
                   "sample": sample},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    rank, world, local_rank = env_rank()
    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local_rank)
    from paper_2509_01928_gb300 import _native as N
    from paper_2509_01928_gb300 import inputs as I
    from paper_2509_01928_gb300.build import build_library

    if rank == 0:
        build_library()
    if world > 1:
        dist.barrier()
    N.load()

    L = args.size
    iters = args.iters
    R = 1
    n = L * L
    t = I.torus_pm1(L, L, seed=SEED + 1000 * rank)
    x0 = I.x0_uniform(n, R, seed=SEED + 1000 * rank)
    prob = N.Problem(t)
    alpha, beta = N.ising_default_params(prob, eta=1.0, method=2)
    handle = N.ising_create(prob, flags=N.FLAG_ASYNC)
    del t
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream
    x0_d = torch.from_numpy(x0).cuda()
    x = torch.empty_like(x0_d)
    E = torch.zeros(1, dtype=torch.int64, device="cuda")
    cut = torch.zeros(1, dtype=torch.int64, device="cuda")
    best = torch.zeros(1, dtype=torch.int32, device="cuda")

    def step(ev_a=None, ev_b=None):
        x.copy_(x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(handle, x, alpha, beta, iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(handle, x, E_int=E, cut_int=cut, best=best, stream=sid)

    for _ in range(args.warmup):
        step()
    N.ising_synchronize(handle, sid)

    gpu_id = None
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local_rank).uuid)
    except Exception:
        gpu_id = None
    sampler = ClockSampler(gpu_id)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t_start.record(stream)
    for k in range(args.steps):
        step(*evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    N.ising_synchronize(handle, sid)
    elapsed = t_start.elapsed_time(t_end) / 1e3
    iter_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    if world > 1:
        tt = torch.tensor([elapsed, iter_s], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        elapsed, iter_s = tt.tolist()
    updates = float(n) * R * iters * args.steps * world
    value = updates / elapsed

    # end to end through the C ABI with pinned host buffers
    xh = torch.from_numpy(x0.copy()).pin_memory()
    Eh = np.zeros(1, np.int64)
    ch = np.zeros(1, np.int64)
    bh = np.zeros(1, np.int32)
    xh_np = xh.numpy()
    n_e2e = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    w0 = time.perf_counter()
    for _ in range(n_e2e):
        N.ising_iterate(handle, xh_np, alpha, beta, iters, stream=sid)      # H2D x, D2H x
        N.ising_energy(handle, xh_np, E_int=Eh, cut_int=ch, best=bh, stream=sid)  # H2D x, D2H E
    e2e_t = time.perf_counter() - w0
    if world > 1:
        tt = torch.tensor([e2e_t], dtype=torch.float64, device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        e2e_t = tt.item()
    e2e_val = float(n) * R * iters * n_e2e * world / e2e_t
    N.ising_destroy(handle)

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    peak, peak_kind = measured_peaks()
    per_launch_s = iter_s / (args.steps * iters)
    alg_bytes = BYTES_PER_SITE * n
    achieved = alg_bytes / per_launch_s / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": recorded_traffic(),
                "kernel": DOMINANT, "peak_kind": peak_kind,
                "algorithmic_bytes_per_launch": alg_bytes}
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        lr = lc = args.ref_size
        u, dt = cpu_oracle_sample(lr, lc, args.cpu_iters)
        cpu = {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"torus {lr}x{lc} int8 +-1, {args.cpu_iters} FP64 DOCH iterations + sign + int64 energy"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (seeded SplitMix64)",
        "config": {"workload": f"torus2d {L}x{L} +-1 int8 couplings, FP32 iterates, R={R}, "
                               f"{iters} DOCH iterations + sign + int64 energy/cut + best replica",
                   "n": n, "replicas": R, "iters": iters, "parallelism": f"replicas-only x{world}",
                   "l2": "inputs larger than L2 (1.2 GB live per step); no flush",
                   "alpha_beta": "Wigner estimate, eta = 1, beta of Eq. alphabeta"},
        "gpu_launches": args.steps * (iters + 3),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * n * 4,
                "d2h_bytes_per_step": n * 4 + 8 + 8 + 4,
                "how": "ising_iterate + ising_energy on pinned host arrays, each step continues from the last"},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "iterate_ms_per_step": 1e3 * iter_s / args.steps,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=10000)
    ap.add_argument("--iters", type=int, default=500)
    ap.add_argument("--ref-size", type=int, default=2048)
    ap.add_argument("--ref-iters", type=int, default=24, help="oracle iterations per reference step")
    ap.add_argument("--cpu-iters", type=int, default=96, help="oracle iterations of the cpu_baseline sample")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
