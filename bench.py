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
# Lattice kernel: one launch performs three DOCH steps (temporal blocking) and reads x (4 B) and
# the right and down couplings (2 B) and writes x (4 B) once per site: 10 B per site per launch,
# 3.3 B per site-update (an iteration count that is not a multiple of 3 ends with one two-step
# pass, which moves the same 10 B per site).
BYTES_PER_SITE = 10
STEPS_PER_LAUNCH = 3
DOMINANT = "torus_f32_r1_vec4_t3"
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "torus_f32_r1_vec4_t3_10000x10000.md")


def env_rank():
    return (int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)),
            int(os.environ.get("LOCAL_RANK", 0)))


def max_over_ranks(vals):
    """Element-wise maximum of per-rank timings over the process group (the whole job is as slow
    as its slowest rank); a single process returns its own values."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return list(vals)
    dev = "cuda" if torch.cuda.is_available() and dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(vals), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def job_rate(units_per_step: float, steps: int, world: int, seconds: float) -> float:
    """Whole-job throughput: every rank processes its own units (weak scaling), timed by the slowest."""
    return units_per_step * steps * world / seconds


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


def _oracle_sample_task(a):
    return cpu_oracle_sample(*a)


def oracle_x_cores(lr: int, lc: int, iters: int):
    """The same oracle sample run as P independent single-threaded processes (one per host core,
    started with spawn), each on its own copy of the sample: an embarrassingly parallel baseline."""
    import multiprocessing as mp
    P = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    with ctx.Pool(P) as pool:
        pool.map(_oracle_sample_task, [(64, 64, 2)] * P)  # start-up and library load, untimed
        w0 = time.perf_counter()
        res = pool.map(_oracle_sample_task, [(lr, lc, iters)] * P)
        wall = time.perf_counter() - w0
    return {"value": sum(u for u, _ in res) / wall, "unit": UNIT, "cores": P, "kind": "oracle x cores",
            "sample": f"{P} processes, each torus {lr}x{lc}, {iters} FP64 DOCH iterations + sign + int64 energy"}


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
        "oracle_x_cores": oracle_x_cores(lr, lc, iters),
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# workloads: one step = one pass of the whole hot path over one batch of input
# ---------------------------------------------------------------------------

class Torus:
    """10^4 x 10^4 periodic lattice, FP32, R = 1, 500 iterations + readout (default)."""

    dominant = DOMINANT
    dtype = "f32"

    def __init__(self, args, rank, N, I, torch):
        self.L, self.iters, self.R = args.size, args.iters, 1
        self.n = self.L * self.L
        t = I.torus_pm1(self.L, self.L, seed=SEED + 1000 * rank)
        self.t = t
        self.x0 = I.x0_uniform(self.n, 1, seed=SEED + 1000 * rank)
        prob = N.Problem(t)
        self.alpha, self.beta = N.ising_default_params(prob, eta=1.0, method=2)
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.E = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.cut = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.best = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        # three steps per lattice launch (the rest in one two-step or one single-step launch)
        self.dominant_launches = self.iters // STEPS_PER_LAUNCH + (1 if self.iters % STEPS_PER_LAUNCH else 0)
        self.launches = self.dominant_launches + 3
        self.config = {"workload": f"torus2d {self.L}x{self.L} +-1 int8 couplings, FP32 iterates, R=1, "
                                   f"{self.iters} DOCH iterations + sign + int64 energy/cut + best replica",
                       "n": self.n, "replicas": 1, "iters": self.iters,
                       "l2": "inputs larger than L2 (1.2 GB live per step); no flush",
                       "alpha_beta": "Wigner estimate, eta = 1, beta of Eq. alphabeta"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_int=self.E, cut_int=self.cut, best=self.best, stream=sid)

    def roofline(self, per_launch_s):
        peak, kind = measured_peaks()
        alg = BYTES_PER_SITE * self.n
        ach = alg / per_launch_s / 1e9
        # the same launch counted per DOCH iteration (10 B per site and iteration, as a
        # one-step pass moves): above 1 by the temporal blocking
        per_iter = BYTES_PER_SITE * self.n * STEPS_PER_LAUNCH / per_launch_s / 1e9 / peak
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": recorded_traffic(), "kernel": self.dominant, "peak_kind": kind,
                "algorithmic_bytes_per_launch": alg, "doch_steps_per_launch": STEPS_PER_LAUNCH,
                "frac_per_iteration_unit": per_iter,
                "note": "three DOCH steps per pass over the lattice: 3.3 B of HBM traffic per site-update; "
                        "the pass is bound by instruction issue, not by HBM"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh_np = self.torch.from_numpy(self.x0.copy()).pin_memory().numpy()
        Eh, ch, bh = np.zeros(1, np.int64), np.zeros(1, np.int64), np.zeros(1, np.int32)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate(self.h, xh_np, self.alpha, self.beta, self.iters, stream=sid)   # H2D x, D2H x
            N.ising_energy(self.h, xh_np, E_int=Eh, cut_int=ch, best=bh, stream=sid)        # H2D x, D2H E
        dt = time.perf_counter() - w0
        return dt, 2 * self.n * 4, self.n * 4 + 8 + 8 + 4, \
            "ising_iterate + ising_energy on pinned host arrays, each step continues from the last"

    def cpu_baseline(self, args):
        """The oracle on a bounded sample of the timed lattice itself: x^(iters) of a 16 x 16 block
        of sites depends only on the sites within `iters` lattice steps, so the oracle runs all
        iterations on that light-cone patch (open boundaries, the lattice's own couplings) -- timed
        as the CPU baseline -- and its block is compared with the GPU's final iterate there."""
        import oracle as O
        from oracle.lattice import light_cone_patch
        size, it = 16, self.iters
        if 2 * it + size > self.L:
            lr = lc = args.ref_size
            u, dt = cpu_oracle_sample(lr, lc, args.cpu_iters)
            return {"value": u / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"torus {lr}x{lc} int8 +-1, {args.cpu_iters} FP64 DOCH iterations"}
        r0 = c0 = 7 * 120 - 8  # straddles a column segment of the multi-step kernels
        J, G = light_cone_patch(self.t, r0, c0, size, it)
        P = size + 2 * it
        t0 = time.perf_counter()
        ref = O.doch(O.Problem(J), self.x0.ravel()[G].astype(np.float64), float(self.alpha[0]),
                     float(self.beta[0]), it).reshape(P, P)
        dt = time.perf_counter() - t0
        blk = ref[it:it + size, it:it + size].ravel()
        sites = G.reshape(P, P)[it:it + size, it:it + size].ravel()
        got = self.x.cpu().numpy().ravel()[sites].astype(np.float64)
        rel = float(np.linalg.norm(got - blk) / np.linalg.norm(blk))
        el = float(np.abs(got - blk).max() / np.abs(blk).max())
        return {"value": P * P * it / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"the light-cone patch ({P}x{P} sites, open boundaries) of a {size}x{size} block of the "
                          f"timed lattice, {it} FP64 DOCH iterations",
                "oracle_match": {"sites": size * size, "iters": it, "rel_err": rel, "max_element_err": el,
                                 "bound": 1e-5, "ok": rel <= 1e-5 and el <= 1e-4,
                                 "what": "the GPU's x^(iters) of the timed run against the oracle at those sites"}}

    def energy(self):
        E, cut = int(self.E.item()), int(self.cut.item())
        return {"E": E, "cut": cut, "E_per_spin": E / self.n, "exact": "int64, sign(x^(iters))"}

    def close(self):
        self.N.ising_destroy(self.h)


class Dense:
    """Dense n = 16384, J = +-1 (BF16, exact), R = 256 BF16 replicas, 1000 iterations on tcgen05."""

    dominant = "dense_tc_kernel"
    dtype = "bf16"

    def __init__(self, args, rank, N, I, torch):
        self.n, self.R, self.iters = args.dense_n, 256, args.dense_iters
        J = I.dense_pm1(self.n, seed=3 + 1000 * rank)
        self.x0 = I.x0_uniform(self.n, self.R, seed=3 + 1000 * rank)
        prob = N.Problem(J)
        self.alpha, self.beta = N.ising_default_params(prob, eta=1.0, method=2)
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0_d = torch.from_numpy(self.x0).to(torch.bfloat16).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.E = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        self.cut = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        self.best = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = self.iters
        self.launches = self.iters + 2 + 4
        self.config = {"workload": f"dense {self.n}x{self.n} +-1 (BF16, exact), R={self.R} BF16 replicas, "
                                   f"{self.iters} DOCH iterations on tcgen05 + exact int64 energy/cut",
                       "n": self.n, "replicas": self.R, "iters": self.iters,
                       "l2": "J held as 67 MB of packed 2-bit codes (L2-resident across iterations); the BF16 "
                             "iterates (8.4 MB each) too; no flush"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_int=self.E, cut_int=self.cut, best=self.best, stream=sid)

    def roofline(self, per_launch_s):
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"]) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1700.0
        flops = 2.0 * self.n * self.n * self.R
        ach = flops / per_launch_s / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant, "peak_kind": "measured (bf16 sustained)",
                "algorithmic_flops_per_launch": flops}

    def e2e(self, n_steps, sid):
        N = self.N
        xh_np = self.x0_d.float().cpu().numpy()
        xh = self.torch.from_numpy(xh_np).to(self.torch.bfloat16).pin_memory()
        Eh = np.zeros(self.R, np.int64)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate(self.h, xh, self.alpha, self.beta, self.iters, stream=sid)
            N.ising_energy(self.h, xh, E_int=Eh, stream=sid)
        dt = time.perf_counter() - w0
        nb = self.n * self.R * 2
        return dt, 2 * nb, nb + 8 * self.R, "ising_iterate + ising_energy on pinned host BF16 arrays"

    def energy(self):
        E = self.E.cpu().numpy().astype(np.float64)
        return {"E_best": float(E.min()), "E_mean": float(E.mean()), "E_std": float(E.std()),
                "replicas": int(E.size), "exact": "int64, sign(x^(iters))"}

    def cpu_baseline(self, args):
        import oracle as O
        from paper_2509_01928_gb300 import inputs as I
        n = 4096
        J = I.dense_pm1(n, seed=3)
        x0 = I.x0_uniform(n, 2, seed=3)
        a, b = O.alpha_beta(J, 1.0, "wigner")
        P = O.Problem(J)
        t0 = time.perf_counter()
        O.doch(P, x0, a, b, 2)
        dt = time.perf_counter() - t0
        return {"value": n * 2 * 2 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"dense {n}x{n} +-1, 2 replicas, 2 FP64 DOCH iterations"}

    def close(self):
        self.N.ising_destroy(self.h)


class Precision:
    """The low-precision form against the plain FP32 form on one dense instance (n = 16384, J = +-1,
    R = 256 replicas from the same seeded start): BF16 iterates with the coupling product on the
    tcgen05 tensor cores (the timed step: 1000 DOCH iterations + exact energy) next to FP32 iterates
    with FP32 products on the CUDA cores. After the timed loop both forms run the same iteration
    count from the same start, recording the integer energies of all replicas every `stride`
    iterations; the line reports each form's spin-updates/s, its final energy distribution (best,
    mean, std over the replicas) and the iterations and time each form needs to bring its mean
    energy within `tol` of the FP32 form's final mean ("equal final energy")."""

    dominant = "dense_tc_kernel"
    dtype = "bf16"

    def __init__(self, args, rank, N, I, torch):
        self.n, self.R, self.iters = args.dense_n, 256, args.dense_iters
        J = I.dense_pm1(self.n, seed=3 + 1000 * rank)
        self.x0 = I.x0_uniform(self.n, self.R, seed=3 + 1000 * rank)
        prob = N.Problem(J)
        self.alpha, self.beta = N.ising_default_params(prob, eta=1.0, method=2)
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0_f32 = torch.from_numpy(self.x0).cuda()
        self.x0_bf16 = self.x0_f32.to(torch.bfloat16)
        self.x0_d = self.x0_bf16
        self.x = torch.empty_like(self.x0_bf16)
        self.E = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = self.iters
        self.launches = self.iters + 2 + 4
        self.stride, self.tol = args.precision_stride, args.precision_tol
        self.config = {"workload": f"dense {self.n}x{self.n} +-1, R={self.R}: BF16 tensor-core form "
                                   f"({self.iters} DOCH iterations + exact energy, timed) against the plain "
                                   f"FP32 CUDA-core form at equal final energy",
                       "n": self.n, "replicas": self.R, "iters": self.iters,
                       "l2": "J held as 67 MB of packed 2-bit codes (L2-resident); no flush"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_bf16)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_int=self.E, stream=sid)

    def _form(self, x0, sid, stream):
        """One uninterrupted run of `iters` iterations (CUDA events) and the energy trajectory of a
        chunked run from the same start (untimed)."""
        N, torch = self.N, self.torch
        x = x0.clone()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        N.ising_iterate(self.h, x, self.alpha, self.beta, self.iters, stream=sid)
        e1.record(stream)
        N.ising_synchronize(self.h, sid)
        sec = e0.elapsed_time(e1) / 1e3
        x = x0.clone()
        E = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        traj = []
        done = 0
        while done < self.iters:
            k = min(self.stride, self.iters - done)
            N.ising_iterate(self.h, x, self.alpha, self.beta, k, stream=sid)
            done += k
            N.ising_energy(self.h, x, E_int=E, stream=sid)
            N.ising_synchronize(self.h, sid)
            traj.append((done, E.cpu().numpy().astype(np.float64)))
        return sec, traj

    def extra(self, sid, stream):
        forms = {}
        for name, x0 in (("bf16_tensor_cores", self.x0_bf16), ("f32_cuda_cores", self.x0_f32)):
            sec, traj = self._form(x0, sid, stream)
            Ef = traj[-1][1]
            forms[name] = {"spin_updates_per_s": self.units / sec, "ms_per_iteration": 1e3 * sec / self.iters,
                           "E_best": float(Ef.min()), "E_mean": float(Ef.mean()), "E_std": float(Ef.std()),
                           "mean_E_trace": [[k, float(e.mean())] for k, e in traj], "_traj": traj,
                           "_sec": sec}
        target = forms["f32_cuda_cores"]["E_mean"]
        thresh = target + self.tol * abs(target)       # energies are negative: within tol above the target
        for f in forms.values():
            hit = next((k for k, e in f.pop("_traj") if e.mean() <= thresh), None)
            sec = f.pop("_sec")
            f["iters_to_equal_energy"] = hit
            f["s_to_equal_energy"] = None if hit is None else sec * hit / self.iters
        b, f = forms["bf16_tensor_cores"], forms["f32_cuda_cores"]
        # the FP32 form on the CUDA cores: 2 n^2 R FP32 flops per iteration against the derived FP32 FMA
        # peak (152 SMs x 128 lanes x 2 flops x 2.07 GHz, the maximum SM clock)
        flops = 2.0 * self.n * self.n * self.R
        f_peak = 152 * 128 * 2 * 2.07e9 / 1e12
        f_ach = flops / (f["ms_per_iteration"] / 1e3) / 1e12
        f["roofline"] = {"bound": "alu", "achieved": f_ach, "peak": f_peak, "unit": "TFLOP/s", "frac": f_ach / f_peak,
                         "kernel": "dense_f32_step", "peak_kind": "derived: FP32 FMA lanes x max SM clock"}
        return {"forms": forms,
                "equal_energy": {"target_mean_E": target, "tol": self.tol,
                                 "mean_E_rel_diff": (b["E_mean"] - f["E_mean"]) / abs(f["E_mean"]),
                                 "best_E_rel_diff": (b["E_best"] - f["E_best"]) / abs(f["E_best"]),
                                 "speedup_at_equal_energy": (f["s_to_equal_energy"] / b["s_to_equal_energy"])
                                 if b["s_to_equal_energy"] and f["s_to_equal_energy"] else None,
                                 "spin_update_rate_ratio": b["spin_updates_per_s"] / f["spin_updates_per_s"]}}

    def roofline(self, per_launch_s):
        peak = float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["bf16_tflops_sustained"]) \
            if os.path.exists(os.path.join(ROOT, "MEASURED_PEAKS.json")) else 1700.0
        flops = 2.0 * self.n * self.n * self.R
        ach = flops / per_launch_s / 1e12
        return {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant, "peak_kind": "measured (bf16 sustained)",
                "algorithmic_flops_per_launch": flops}

    def e2e(self, n_steps, sid):
        return Dense.e2e(self, n_steps, sid)

    def energy(self):
        return Dense.energy(self)

    def cpu_baseline(self, args):
        return Dense.cpu_baseline(self, args)

    def close(self):
        self.N.ising_destroy(self.h)


class Batched:
    """512 uneven instances (n ~ U[500, 20000], d-regular d ~ U{3..10}, J ~ N(0,1) FP32,
    h ~ N(0, 0.1)), R = 16, 2000 iterations in one persistent launch (each instance's replica
    groups resident in shared memory)."""

    dominant = "batched_resident"
    dtype = "f32"

    def __init__(self, args, rank, N, I, torch):
        ns, ds = I.batched_sizes(args.batch_count, 500, 20000, 3, 10, seed=4 + 1000 * rank)
        gs = [I.regular_gauss(int(n), int(d), seed=5000 + b + 100000 * rank) for b, (n, d) in enumerate(zip(ns, ds))]
        hs = [I.field_gauss(g.n, 0.1, seed=7000 + b + 100000 * rank) for b, g in enumerate(gs)]
        off = np.cumsum([0] + [g.n for g in gs]).astype(np.int64)
        nz = np.cumsum([0] + [g.nnz for g in gs])
        rp = np.concatenate([[0]] + [g.row_ptr[1:] + z for g, z in zip(gs, nz[:-1])])
        col = np.concatenate([g.col + o for g, o in zip(gs, off[:-1])]).astype(np.int32)
        val = np.concatenate([g.val for g in gs]).astype(np.float32)
        self.nnz = int(nz[-1])
        h = np.concatenate(hs).astype(np.float32)
        self.n, self.R, self.iters, self.B = int(off[-1]), 16, args.batch_iters, len(gs)
        prob = N.Problem(I.CSR(self.n, rp, col, val), h, off)
        self.alpha, self.beta = N.ising_default_params(prob, eta=1.0, method=0)
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0 = I.x0_uniform(self.n, self.R, seed=4 + 1000 * rank)
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.E = torch.zeros((self.B, self.R), dtype=torch.float64, device="cuda")
        self.best = torch.zeros(self.B, dtype=torch.int32, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = 1
        self.launches = 1 + 3
        self.config = {"workload": f"batched {self.B} instances, n in [500, 20000] (sum {self.n}), random "
                                   f"d-regular d in 3..10, J ~ N(0,1) FP32, h ~ N(0,0.1), R={self.R}, "
                                   f"{self.iters} iterations in one persistent launch (replica groups resident in shared memory) + FP64 energy",
                       "n": self.n, "instances": self.B, "replicas": self.R, "iters": self.iters,
                       "l2": "live set ~1.1 GB (> L2); per-instance state L2-resident during its run"}
        # first call tunes the launch shape and captures the graph
        self.x.copy_(self.x0_d)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, 4, n_instances=self.B)
        N.ising_synchronize(self.h)

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid, n_instances=self.B)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_f64=self.E, best=self.best, stream=sid)

    def roofline(self, per_launch_s):
        peak, kind = measured_peaks()
        # per iteration, streamed: col 4 B + val 4 B per entry, x read + write, h, row_ptr
        per_iter = 8 * self.nnz + 2 * self.n * self.R * 4 + self.n * 4 + self.n * 8
        alg = per_iter * self.iters
        ach = alg / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant, "peak_kind": kind,
                "algorithmic_bytes_per_launch": alg,
                "note": "bytes of an iteration streamed from HBM (CSR entries, x read and write, h); "
                        "the kernel keeps each (instance, replica group) of x in shared memory for all "
                        "iterations and re-reads only the couplings, from L2"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh = self.torch.from_numpy(self.x0.copy()).pin_memory().numpy()
        Eh = np.zeros((self.B, self.R))
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate(self.h, xh, self.alpha, self.beta, self.iters, stream=sid, n_instances=self.B)
            N.ising_energy(self.h, xh, E_f64=Eh, stream=sid)
        dt = time.perf_counter() - w0
        nb = self.n * self.R * 4
        return dt, 2 * nb, nb + 8 * self.B * self.R, "ising_iterate + ising_energy on pinned host arrays"

    def cpu_baseline(self, args):
        import oracle as O
        from paper_2509_01928_gb300 import inputs as I
        g = I.regular_gauss(10000, 6, seed=5)
        h = I.field_gauss(g.n, 0.1, seed=6)
        x0 = I.x0_uniform(g.n, 16, seed=5)
        a, b = O.alpha_beta(g, 1.0, "eig")
        P = O.Problem(g, h)
        t0 = time.perf_counter()
        O.doch(P, x0, a, b, 200)
        dt = time.perf_counter() - t0
        return {"value": g.n * 16 * 200 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "one instance n = 10000, 6-regular, Gaussian J, h, R = 16, 200 FP64 iterations"}

    def close(self):
        self.N.ising_destroy(self.h)


class Backward:
    """Adjoint: 3-regular n = 1e5, +-1, R = 64, 200 FP32 iterations, checkpoint every 20."""

    dominant = "adjoint_step_kernel"
    dtype = "f32"

    def __init__(self, args, rank, N, I, torch):
        g = I.regular_pm1(100000, 3, seed=5 + 1000 * rank)
        self.n, self.R, self.iters, self.ckpt = g.n, 64, 200, 20
        prob = N.Problem(g)
        a, self.beta = N.ising_default_params(prob, eta=1.0, method=2)
        self.alpha = np.full(self.iters, a[0])
        self.beta = float(self.beta[0])
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0 = I.x0_uniform(self.n, self.R, seed=5 + 1000 * rank)
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.ga = torch.zeros(self.iters, dtype=torch.float64, device="cuda")
        self.gx = torch.zeros_like(self.x0_d)
        self.loss = torch.zeros(1, dtype=torch.float64, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = self.iters
        self.launches = 3 * self.iters + 4
        self.config = {"workload": f"adjoint: random 3-regular n=1e5 +-1, R=64, {self.iters} FP32 iterations, "
                                   f"checkpoint every {self.ckpt}: loss + dL/dalpha[200] + dL/dx0",
                       "n": self.n, "replicas": self.R, "iters": self.iters,
                       "metric_note": "forward spin-updates per second of the whole gradient computation "
                                      "(forward, recompute and adjoint)",
                       "l2": "x 25.6 MB L2-resident"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        if ev_a is not None:
            ev_a.record(stream)
        self.N.ising_backward(self.h, self.x0_d, self.alpha, self.beta, self.iters, self.ckpt,
                              grad_alpha=self.ga, grad_x0=self.gx, loss=self.loss, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)

    def roofline(self, per_launch_s):
        # per step index k the call runs a forward step, a recompute step and an adjoint step; unique
        # bytes: forward and recompute read and write x (2 n R 4 B each) and read the CSR arrays; the
        # adjoint reads w^k and x^k and writes w^(k-1) (3 n R 4 B) and reads the CSR arrays.
        # The 25.6 MB iterates stay in L2, so this is the HBM-equivalent rate of the whole step triple.
        peak, kind = measured_peaks()
        nnz = 3 * self.n
        csr = nnz * (4 + 1) + (self.n + 1) * 8
        xb = self.n * self.R * 4
        alg = 2 * (2 * xb + csr) + (3 * xb + csr)
        ach = alg / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "kernel": "csr_step_kernel (forward, recompute) + adjoint_step_kernel",
                "peak_kind": kind, "algorithmic_bytes_per_launch": alg,
                "launch": "one step index: forward step + recompute step + adjoint step",
                "note": "iterates L2-resident: an HBM-equivalent rate of unique bytes"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh = self.torch.from_numpy(self.x0.copy()).pin_memory().numpy()
        ga = np.zeros(self.iters)
        gx = np.zeros_like(self.x0)
        loss = np.zeros(1)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_backward(self.h, xh, self.alpha, self.beta, self.iters, self.ckpt, grad_alpha=ga,
                             grad_x0=gx, loss=loss, stream=sid)
        dt = time.perf_counter() - w0
        nb = self.n * self.R * 4
        return dt, nb, nb + 8 * (self.iters + 1), "ising_backward on pinned host x0, host gradients"

    def cpu_baseline(self, args):
        import oracle as O
        from paper_2509_01928_gb300 import inputs as I
        g = I.regular_pm1(100000, 3, seed=5)
        x0 = I.x0_uniform(g.n, 2, seed=5)
        a, b = O.alpha_beta(g, 1.0, "wigner")
        t0 = time.perf_counter()
        O.backward(O.Problem(g), x0, np.full(self.iters, a), b, self.iters)
        dt = time.perf_counter() - t0
        return {"value": g.n * 2 * self.iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"adjoint of {self.iters} FP64 steps, n = 1e5 3-regular, 2 replicas"}

    def close(self):
        self.N.ising_destroy(self.h)


class Er800:
    """Plain method, FP64: Erdos-Renyi n = 800, p = 0.06, +-1, R = 8, 1000 iterations."""

    dominant = "csr_fused_kernel"
    dtype = "f64"

    def __init__(self, args, rank, N, I, torch):
        g = I.erdos_renyi_pm1(800, 0.06, seed=1 + 1000 * rank)
        self.n, self.R, self.iters = g.n, 8, 1000
        self.nnz = int(g.row_ptr[-1])
        prob = N.Problem(g)
        self.alpha, self.beta = N.ising_default_params(prob, eta=1.0, method=1)
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0 = I.x0_uniform(self.n, self.R, seed=2 + 1000 * rank, dtype=np.float64)
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.E = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        self.cut = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        self.best = torch.zeros(1, dtype=torch.int32, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = 1
        self.launches = 1 + 3
        self.config = {"workload": "plain method FP64: Erdos-Renyi n=800 p=0.06 +-1, R=8, 1000 iterations "
                                   "(one launch, iterate in shared memory) + int64 energy/cut + best replica",
                       "n": self.n, "replicas": self.R, "iters": self.iters, "l2": "on-chip problem"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_int=self.E, cut_int=self.cut, best=self.best, stream=sid)

    def roofline(self, per_launch_s):
        # FP64 arithmetic of the 1000 steps in the one launch: a multiply-add per stored coupling and
        # replica, and alpha x, the scale and the cube root's argument per spin and replica (cube root
        # not counted); against the nominal dense FP64 rate of the part (1.25 TFLOP/s). One CTA per
        # replica (8 of 152 SMs) holds the iterate in shared memory: the launch is latency-bound.
        nnz = self.nnz
        flops = self.iters * self.R * (2.0 * nnz + 3.0 * self.n)
        ach = flops / per_launch_s / 1e9
        peak = 1250.0
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "GFLOP/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant, "peak_kind": "nominal FP64 (1.25 TFLOP/s)",
                "algorithmic_flops_per_launch": flops,
                "note": "one CTA per replica on 8 of 152 SMs; latency-bound"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh = self.x0.copy()
        Eh = np.zeros(self.R, np.int64)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate(self.h, xh, self.alpha, self.beta, self.iters, stream=sid)
            N.ising_energy(self.h, xh, E_int=Eh, stream=sid)
        dt = time.perf_counter() - w0
        nb = self.n * self.R * 8
        return dt, 2 * nb, nb + 8 * self.R, "ising_iterate + ising_energy on host arrays"

    def cpu_baseline(self, args):
        import oracle as O
        from paper_2509_01928_gb300 import inputs as I
        g = I.erdos_renyi_pm1(800, 0.06, seed=1)
        x0 = I.x0_uniform(g.n, 8, seed=2, dtype=np.float64)
        a, b = O.alpha_beta(g, 1.0, "eig")
        t0 = time.perf_counter()
        O.doch(O.Problem(g), x0, a, b, 1000)
        dt = time.perf_counter() - t0
        return {"value": g.n * 8 * 1000 / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": "the whole workload: n = 800, R = 8, 1000 FP64 iterations"}

    def close(self):
        self.N.ising_destroy(self.h)


class Adoch:
    """ADOCH (Algorithm 2) on the 10^4 x 10^4 lattice, FP32, R = 1, q = 5, 100 steps per timed step."""

    dominant = "adoch step (adoch_lattice<2> + adoch_lattice_bound + adoch_decide)"
    dtype = "f32"

    def __init__(self, args, rank, N, I, torch):
        self.L, self.iters, self.R, self.q = args.size, args.adoch_iters, 1, 5
        self.n = self.L * self.L
        t = I.torus_pm1(self.L, self.L, seed=SEED + 1000 * rank)
        self.t = t
        self.x0 = I.x0_uniform(self.n, 1, seed=SEED + 1000 * rank)
        prob = N.Problem(t)
        self.alpha, self.beta = N.ising_default_params(prob, eta=1.0, method=2)
        self.h = N.ising_create(prob, flags=N.FLAG_ASYNC)
        self.N, self.torch = N, torch
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.acc = torch.zeros((self.iters, 1), dtype=torch.int8, device="cuda")
        self.E = torch.zeros(1, dtype=torch.int64, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = self.iters  # one ADOCH step = pass + decide + update
        # step 0: pass + decide; steps 1..N-1: one pass (update and next terms) + boundary edges +
        # decide; the last step: update only; readout: row_reduce + energy_finish
        self.launches = 3 * self.iters + 2
        self.config = {"workload": f"ADOCH (Algorithm 2) on the torus2d {self.L}x{self.L} +-1 int8 lattice, FP32, "
                                   f"R=1, q={self.q}, {self.iters} steps + sign + int64 energy",
                       "n": self.n, "replicas": 1, "iters": self.iters, "q": self.q,
                       "l2": "inputs larger than L2 (2 GB live per step); no flush",
                       "alpha_beta": "Wigner estimate, eta = 1, beta of Eq. alphabeta"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate_adoch(self.h, self.x, self.alpha, self.beta, self.iters, self.q, accepted=self.acc,
                              stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_int=self.E, stream=sid)

    def roofline(self, per_launch_s):
        peak, kind = measured_peaks()
        # per step and site: one pass reads x^k, x^(k-1) and the couplings (10 B) and writes x^(k+1)
        # (4 B), forming from the new values the H terms of the next step (plus an edge pass over
        # the ~1 % of sites on warp and strip boundaries, not counted)
        alg = 14 * self.n
        ach = alg / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant, "peak_kind": kind,
                "algorithmic_bytes_per_launch": alg, "launch": "one ADOCH step (3 kernels)"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh = self.torch.from_numpy(self.x0.copy()).pin_memory().numpy()
        Eh = np.zeros(1, np.int64)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate_adoch(self.h, xh, self.alpha, self.beta, self.iters, self.q, stream=sid)
            N.ising_energy(self.h, xh, E_int=Eh, stream=sid)
        dt = time.perf_counter() - w0
        return dt, 2 * self.n * 4, self.n * 4 + 8, "ising_iterate_adoch + ising_energy on pinned host arrays"

    def cpu_baseline(self, args):
        import oracle as O
        from paper_2509_01928_gb300 import inputs as I
        lr = lc = 1024
        iters = 60
        t = I.torus_pm1(lr, lc, seed=SEED)
        x0 = I.x0_uniform(t.n, 1, seed=SEED)
        P = O.Problem(t)
        a, b = O.alpha_beta(t, eta=1.0, method="wigner")
        t0 = time.perf_counter()
        O.adoch(P, x0, a, b, iters, self.q)
        dt = time.perf_counter() - t0
        return {"value": t.n * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"ADOCH on a torus {lr}x{lc} int8 +-1, {iters} FP64 steps, q = {self.q}"}

    def close(self):
        self.N.ising_destroy(self.h)


class S5:
    """Algorithm S5 matrix generated on the device (n = 1e5, p = 0.1 %, ~1e7 couplings), parameters on
    the device, then 500 FP32 DOCH steps with R = 16 on the CSR path."""

    dominant = "csr_step_kernel"
    dtype = "f32"

    def __init__(self, args, rank, N, I, torch):
        self.n, self.p, self.R, self.iters = args.s5_n, args.s5_p, 16, args.s5_iters
        self.N, self.torch = N, torch
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        self.h = N.ising_create_s5(self.n, self.p, 17 + 1000 * rank, flags=N.FLAG_ASYNC)
        t1 = time.perf_counter()
        self.alpha, self.beta = N.ising_params_device(self.h, eta=1.0, method=2)
        t2 = time.perf_counter()
        rp, _, _ = N.ising_csr_export(self.h)
        self.nnz = int(rp[-1])
        self.x0 = I.x0_uniform(self.n, self.R, seed=18 + 1000 * rank)
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.E = torch.zeros(self.R, dtype=torch.int64, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = self.iters
        self.launches = self.iters + 3
        self.config = {"workload": f"Algorithm S5 n={self.n} p={self.p}% (9-bit couplings, {self.nnz} stored "
                                   f"entries) generated on the device, Wigner parameters on the device, R={self.R} "
                                   f"FP32, {self.iters} DOCH steps + sign + int64 energy",
                       "n": self.n, "nnz": self.nnz, "replicas": self.R, "iters": self.iters,
                       "generate_ms": 1e3 * (t1 - t0), "params_ms": 1e3 * (t2 - t1),
                       "l2": "iterate (6.4 MB) L2-resident; couplings (80 MB) streamed; no flush"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_int=self.E, stream=sid)

    def roofline(self, per_launch_s):
        peak, kind = measured_peaks()
        # per step from HBM: col 4 B + val 4 B per stored entry, x read and written once
        alg = 8 * self.nnz + 2 * self.n * self.R * 4
        ach = alg / per_launch_s / 1e9
        return {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant, "peak_kind": kind, "algorithmic_bytes_per_launch": alg,
                "note": "the neighbour gathers (nnz x R x 4 B per step) are served from L2 and not counted"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh = self.torch.from_numpy(self.x0.copy()).pin_memory().numpy()
        Eh = np.zeros(self.R, np.int64)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate(self.h, xh, self.alpha, self.beta, self.iters, stream=sid)
            N.ising_energy(self.h, xh, E_int=Eh, stream=sid)
        dt = time.perf_counter() - w0
        nb = self.n * self.R * 4
        return dt, 2 * nb, nb + 8 * self.R, "ising_iterate + ising_energy on pinned host arrays"

    def cpu_baseline(self, args):
        import oracle as O
        from oracle import matrices as M
        from paper_2509_01928_gb300 import inputs as I
        n, p, iters = 20000, 0.1, 200
        J = M.s5_csr(n, p, seed=17)
        x0 = I.x0_uniform(n, self.R, seed=18, dtype=np.float64)
        a, b = O.alpha_beta(J, eta=1.0, method="wigner")
        P = O.Problem(J)
        t0 = time.perf_counter()
        O.doch(P, x0, a, b, iters)
        dt = time.perf_counter() - t0
        return {"value": n * self.R * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"Algorithm S5 n={n} p={p}%, R={self.R}, {iters} FP64 DOCH steps"}

    def close(self):
        self.N.ising_destroy(self.h)


class Proc:
    """Procedural dense couplings J_ij = sin(i j + 100) of Supplementary Note 9 (the fully connected
    benchmark matrix, never stored), n = 1e6, one replica, FP32: 10 DOCH steps + sign + energy."""

    dominant = "proc_sym"
    dtype = "f32"
    OPS_PER_COUPLING = 10  # phase add 1, |s| 1, convert 1, fold 1, square 1, polynomial 4, sign 1
    # one replica: the symmetric product generates each unordered pair once (10 / 2 per coupling)
    # and multiply-adds it twice; wider replica groups generate every coupling (10 per coupling)

    def __init__(self, args, rank, N, I, torch):
        self.n, self.R, self.iters = args.proc_n, 1, args.proc_iters
        self.N, self.torch = N, torch
        t0 = time.perf_counter()
        self.h = N.ising_create_procedural(self.n, 100, flags=N.FLAG_ASYNC)
        t1 = time.perf_counter()
        self.alpha, self.beta = N.ising_params_device(self.h, eta=1.0, method=2)
        t2 = time.perf_counter()
        self.x0 = I.x0_uniform(self.n, self.R, seed=SEED + 1000 * rank)
        self.x0_d = torch.from_numpy(self.x0).cuda()
        self.x = torch.empty_like(self.x0_d)
        self.E = torch.zeros(self.R, dtype=torch.float64, device="cuda")
        self.units = float(self.n) * self.R * self.iters
        self.dominant_launches = self.iters
        # per DOCH step: max |x|, symmetric product, finish; readout: spins, product, quadratic form
        self.launches = 3 * self.iters + 3
        self.config = {"workload": f"procedural dense J_ij = sin(ij + 100), n={self.n} (n^2 = {self.n ** 2:.1e} "
                                   f"couplings generated per product), R={self.R}, FP32, {self.iters} DOCH steps "
                                   f"+ sign + FP64 energy",
                       "n": self.n, "replicas": self.R, "iters": self.iters,
                       "create_ms": 1e3 * (t1 - t0), "params_ms": 1e3 * (t2 - t1),
                       "l2": f"compute bound; the iterate ({self.n * self.R * 4 / 1e6:.0f} MB) is L2-resident; "
                             "no flush",
                       "alpha_beta": "Wigner estimate on the device, eta = 1, beta of Eq. alphabeta"}

    def step(self, sid, stream, ev_a=None, ev_b=None):
        N = self.N
        self.x.copy_(self.x0_d)
        if ev_a is not None:
            ev_a.record(stream)
        N.ising_iterate(self.h, self.x, self.alpha, self.beta, self.iters, stream=sid)
        if ev_b is not None:
            ev_b.record(stream)
        N.ising_energy(self.h, self.x, E_f64=self.E, stream=sid)

    def roofline(self, per_launch_s):
        # ALU bound: lane operations per coupling (generation + one FMA per replica) against
        # 152 SMs x 128 FP32/INT32 lanes x 2.07 GHz (the maximum SM clock)
        gen = self.OPS_PER_COUPLING / 2 if self.R == 1 else self.OPS_PER_COUPLING
        ops = float(self.n) ** 2 * (gen + self.R)
        ach = ops / per_launch_s / 1e9
        peak = 152 * 128 * 2.07
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "Gop/s", "frac": ach / peak,
                "traffic": None, "kernel": self.dominant,
                "peak_kind": "derived: 152 SMs x 128 lanes x 2.07 GHz max SM clock",
                "algorithmic_ops_per_launch": ops, "couplings_per_s": float(self.n) ** 2 / per_launch_s,
                "launch": "one coupling product (proc_maxabs + proc_sym over all work units + proc_sym_finish)"}

    def e2e(self, n_steps, sid):
        N = self.N
        xh = self.torch.from_numpy(self.x0.copy()).pin_memory().numpy()
        Eh = np.zeros(self.R)
        w0 = time.perf_counter()
        for _ in range(n_steps):
            N.ising_iterate(self.h, xh, self.alpha, self.beta, self.iters, stream=sid)
            N.ising_energy(self.h, xh, E_f64=Eh, stream=sid)
        dt = time.perf_counter() - w0
        nb = self.n * self.R * 4
        return dt, 2 * nb, nb + 8 * self.R, "ising_iterate + ising_energy on pinned host arrays"

    def cpu_baseline(self, args):
        import oracle as O
        from oracle import matrices as M
        from paper_2509_01928_gb300 import inputs as I
        n, iters = 4000, 300
        J = M.procedural_sin(n, 100)
        x0 = I.x0_uniform(n, self.R, seed=SEED, dtype=np.float64)
        a, b = O.alpha_beta(J, eta=1.0, method="wigner")
        P = O.Problem(J)
        t0 = time.perf_counter()
        O.doch(P, x0, a, b, iters)
        dt = time.perf_counter() - t0
        return {"value": n * self.R * iters / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
                "sample": f"procedural sin(ij + 100) n={n} held as a stored FP64 matrix, R={self.R}, "
                          f"{iters} FP64 DOCH steps"}

    def close(self):
        self.N.ising_destroy(self.h)


WORKLOADS = {"torus": Torus, "dense": Dense, "batched": Batched, "backward": Backward, "er800": Er800,
             "adoch": Adoch, "s5": S5, "proc": Proc, "precision": Precision}


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

    wl = WORKLOADS[args.workload](args, rank, N, I, torch)
    stream = torch.cuda.current_stream()
    sid = stream.cuda_stream

    for _ in range(args.warmup):
        wl.step(sid, stream)
    N.ising_synchronize(wl.h, sid)

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
        wl.step(sid, stream, *evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = sampler.stop()
    N.ising_synchronize(wl.h, sid)
    elapsed = t_start.elapsed_time(t_end) / 1e3
    dom_s = sum(a.elapsed_time(b) for a, b in evs) / 1e3
    elapsed, dom_s = max_over_ranks([elapsed, dom_s])
    value = job_rate(wl.units, args.steps, world, elapsed)

    # end to end through the C ABI with pinned host buffers
    n_e2e = max(1, min(args.steps, 3))
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    e2e_t, h2d, d2h, how = wl.e2e(n_e2e, sid)
    (e2e_t,) = max_over_ranks([e2e_t])
    e2e_val = job_rate(wl.units, n_e2e, world, e2e_t)
    extra = wl.extra(sid, stream) if hasattr(wl, "extra") else None
    wl.close()

    if rank != 0:
        if world > 1:
            dist.destroy_process_group()
        return

    per_launch_s = dom_s / (args.steps * wl.dominant_launches)
    roofline = wl.roofline(per_launch_s)
    cpu = wl.cpu_baseline(args) if (world == 1 and not args.no_cpu_baseline) else None
    config = dict(wl.config)
    config["parallelism"] = f"replicas-only x{world}"
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": wl.dtype, "data": "synthetic (seeded SplitMix64)",
        "config": config,
        "gpu_launches": args.steps * wl.launches,
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "how": how},
        "roofline": roofline,
        "cpu_baseline": cpu,
        "clocks": clocks,
        "dominant_ms_per_step": 1e3 * dom_s / args.steps,
    }
    if extra is not None:
        line["precision"] = extra
    if hasattr(wl, "energy"):
        line["energy"] = wl.energy()
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
    ap.add_argument("--workload", default="torus", choices=sorted(WORKLOADS),
                    help="torus (default: 10^4 x 10^4 lattice), dense (16384 x 256 on tcgen05), "
                         "batched (512 uneven instances), backward (adjoint, n = 1e5), er800 (FP64), "
                         "adoch (Algorithm 2 on the 10^4 x 10^4 lattice), s5 (Algorithm S5 matrix generated on "
                         "the device, n = 1e5), proc (procedural dense sin(ij + 100), n = 1e6), precision (dense 16384 x 256: "
                         "BF16 tensor-core form against the plain FP32 form at equal final energy)")
    ap.add_argument("--dense-n", type=int, default=16384)
    ap.add_argument("--dense-iters", type=int, default=1000)
    ap.add_argument("--batch-count", type=int, default=512)
    ap.add_argument("--batch-iters", type=int, default=2000)
    ap.add_argument("--adoch-iters", type=int, default=100)
    ap.add_argument("--s5-n", type=int, default=100000)
    ap.add_argument("--s5-p", type=float, default=0.1)
    ap.add_argument("--s5-iters", type=int, default=500)
    ap.add_argument("--proc-n", type=int, default=1000000)
    ap.add_argument("--proc-iters", type=int, default=10)
    ap.add_argument("--precision-stride", type=int, default=50, help="iterations between energy readouts")
    ap.add_argument("--precision-tol", type=float, default=0.005, help="relative tolerance of equal final energy")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
