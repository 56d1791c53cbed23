#!/usr/bin/env python3
"""Benchmark: Lanczos steps on the s = 1/2 J1-J2 ring N = 32 (J1 = -1, J2 = -0.5),
sector M = 0 (dim C(32,16) = 601,080,390), FP64 vectors.

A step is one full Lanczos iteration through the C ABI: the row matvec with its fused
epilogue (u = H v_j - beta v_{j-1}, alpha_j partials), the alpha reduction, the update
(w = u - alpha v_j, |w|^2 partials) and the beta reduction.  The metric is Gnnz/s: the
non-zero matrix elements one product applies (20,456,122,950 here) per step, over the
timed steps.  The vectors (2 x 4.8 GB) are far larger than L2, so no L2 flush is needed.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload j1j2_ring32|j1j2_ring32_flip|ring24_randJ|ring24_grad|ring16 ...]

--impl reference times the CPU oracle (test infrastructure, the only baseline: the paper
ships no code) on the host cores, on bounded row samples of the same workload.
Under torchrun (N > 1) every rank runs an independent replica (the sector product needs
no exchange between replicas); value = all ranks' work / the slowest rank's time.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "H(M) matvec Gnnz/s"
UNIT = "Gnnz/s"

WORKLOADS = {
    # name: nnz per product = dim + number of allowed exchange hops.  For s = 1/2 at
    # M = 0 every bond connects C(N-2, N/2-1) states in each direction, so
    # nnz = C(N, N/2) + 2 n_bonds C(N-2, N/2-1).
    "j1j2_ring32": 20456122950,
    # the spin-flip +1 block of the same sector: the representatives are the first half of
    # the rows, and no two exchanges of a row fold onto one column (N >= 6), so half the nnz
    "j1j2_ring32_flip": 10228061475,
    "j1j2_ring28": 1204983800,
    "ring24_randJ": 70425628,
    "ring16": 122694,
    # finite-temperature Lanczos: nnz counted per sector and per executed vector-step
    "ftlm_ring24": None,
    # differentiation (config 4): one step = y = H x through the autograd function and its
    # backward (dL/dx = H g, dL/dJ by the bond-correlation kernel): 3 x nnz of the sector
    "ring24_grad": 70425628,
    # s = 1 random 4-regular graph, N = 20 (FP32 vectors by default); nnz from count_nnz
    "s1_rrg20": None,
    # Arnoldi with full re-orthogonalisation on the N = 24 J1-J2 ring: one step = one whole
    # 60-step run; Gnnz/s counts its products (48 bonds, M = 0)
    "arnoldi_ring24": 2704156 + 2 * 48 * 705432,
    # momentum block k = 0 of the default ring sector (18.8 million states); nnz = the terms
    # its product processes (count_nnz on the momentum basis)
    "j1j2_ring32_k0": None,
}
DEFAULT_DTYPE = {"s1_rrg20": "f32"}
PARITY = {"j1j2_ring32_flip": 1}     # spin-flip block (basis_build_flip) of the workload's sector
MOMENTUM = {"j1j2_ring32_k0": 0}     # momentum block (basis_build_momentum) of the workload's sector

# bytes one product must move at minimum: read x once, write y once (FP64)
ALGO_BYTES_PER_ROW = 16


def instance(name):
    from paper_0706_3293_gb300 import workloads as W
    return {"j1j2_ring32": W.j1j2_ring32, "j1j2_ring32_flip": W.j1j2_ring32, "j1j2_ring32_k0": W.j1j2_ring32,
            "j1j2_ring28": lambda: W.j1j2_ring(28),
            "ring24_randJ": W.ring24_random_j, "ring24_grad": W.ring24_random_j, "ring16": W.ring16,
            "ftlm_ring24": W.ftlm_ring24, "arnoldi_ring24": W.arnoldi_ring24,
            "s1_rrg20": W.s1_random_graph}[name]()


def workload_name(inst, parity, momentum=None):
    name = inst.name + (f"_flip{parity:+d}" if parity else "")
    return name + ("" if momentum is None else ("_k0" if momentum == 0 else "_kpi"))


def sector_nnz_s12(n_sites: int, n_bonds: int, A: int) -> int:
    """nnz of one s = 1/2 sector: C(N, A) diagonal elements plus, for every bond, the
    2 C(N-2, A-1) states whose two spins differ (each has one exchange)."""
    import math
    return math.comb(n_sites, A) + (2 * n_bonds * math.comb(n_sites - 2, A - 1) if A >= 1 else 0)


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(value: float, ws: int, device="cpu") -> float:
    """The slowest rank's time: all_reduce(MAX) over the process group (identity for one
    process).  device: where the reduction tensor lives (cuda for NCCL, cpu for gloo)."""
    if ws <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def kernel_source_hash() -> str:
    h = hashlib.sha256()
    d = os.path.join(ROOT, "paper_0706_3293_gb300", "csrc")
    for f in sorted(os.listdir(d)):
        if f.endswith((".cu", ".cuh")):
            h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def read_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        try:
            d = json.load(open(p))
            return float(d["hbm_gbs"]), "measured"
        except Exception:
            pass
    return 6800.0, "fallback"


def read_traffic(kernel: str, workload: str):
    """Per-launch DRAM bytes of the kernel from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.txt")
    if not os.path.exists(p):
        return None
    cur = kernel_source_hash()
    for line in open(p):
        parts = line.split()
        if len(parts) >= 4 and parts[0] == kernel and parts[1] == workload and parts[3] == cur:
            return float(parts[2])
    return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.rows = []
        self.proc = None
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        def rd():
            for line in self.proc.stdout:
                self.rows.append([c.strip() for c in line.split(",")])
        self.thread = threading.Thread(target=rd, daemon=True)
        self.thread.start()

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm = []
        mx = None
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1]))
                mx = float(r[2])
                for k, nm in enumerate(names):
                    if r[4 + k].lower().startswith("active"):
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_vector(ob, inst, parity):
    """The oracle's start vector for the workload's product: the sector vector, or for a
    spin-flip block the sector vector [x, parity reversed(x)] its representatives stand for
    (the block's rows are the first half of the sector's).  Returns (vector, rows)."""
    import numpy as np
    import oracle
    if not parity:
        return oracle.start_uniform(inst.seed, ob.dim), ob.dim
    xr = oracle.start_uniform(inst.seed, ob.dim // 2)
    return np.concatenate([xr, parity * xr[::-1]]), ob.dim // 2


def cpu_baseline(inst, nnz_total, target_s=15.0, parity=0):
    """The oracle's row matvec on a bounded contiguous sample of rows, all host cores."""
    import numpy as np
    import oracle
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bonds = oracle.Bonds(inst.u, inst.v, inst.J)
    x, rows = oracle_vector(ob, inst, parity)
    mid = rows // 3
    pilot = min(rows, 200000)
    t0 = time.perf_counter()
    ob.matvec_rows(bonds, x, mid if mid + pilot <= rows else 0, (mid if mid + pilot <= rows else 0) + pilot)
    rate = pilot / max(time.perf_counter() - t0, 1e-6)
    n = int(min(rows, max(pilot, rate * target_s)))
    r0 = min(mid, rows - n)
    t0 = time.perf_counter()
    ob.matvec_rows(bonds, x, r0, r0 + n)
    dt = time.perf_counter() - t0
    nnz = ob.count_nnz(bonds, r0, r0 + n)
    del x
    return {"value": nnz / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"rows [{r0}, {r0 + n}) of one FP64 product ({n} of {rows} rows, "
                      f"{nnz} nnz, {dt:.1f} s)"}


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    inst = instance(args.workload)
    if args.workload in MOMENTUM:
        print(json.dumps({"impl": "reference", "unavailable": "the oracle builds momentum blocks densely, "
                          "for small N only; no bounded sample of this workload exists"}))
        return 0
    if args.workload == "arnoldi_ring24":
        # one step = the oracle's Arnoldi on the first 6 steps of the run (bounded sample)
        nnz = WORKLOADS[args.workload]
        for _ in range(args.warmup):
            arnoldi_oracle_rate(inst, nnz, 2)
        vals, tsum = [], 0.0
        for _ in range(args.steps):
            cb, dt = arnoldi_oracle_rate(inst, nnz, 6)
            vals.append(cb["value"])
            tsum += dt
        val = float(np.mean(vals))
        cb["value"] = val
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": tsum / args.steps * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": inst.name, "n_sites": inst.n_sites,
                                              "step": "the first 6 Arnoldi steps"},
               "cpu_baseline": cb,
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return 0
    if args.workload == "ring24_grad":
        nnz = WORKLOADS[args.workload]
        for _ in range(args.warmup):
            grad_oracle_rate(inst, nnz, 1)
        cb = grad_oracle_rate(inst, nnz, args.steps)
        val = cb["value"]
        out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": 3 * nnz / (val * 1e9) * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
               "data": "synthetic", "config": {"workload": inst.name + "_grad", "n_sites": inst.n_sites,
                                              "products_per_step": 3},
               "cpu_baseline": cb,
               "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(out))
        return 0
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bonds = oracle.Bonds(inst.u, inst.v, inst.J)
    parity = PARITY.get(args.workload, 0)
    x, rows = oracle_vector(ob, inst, parity)
    # one step = one oracle product over a bounded row sample sized to ~3 s
    pilot = min(rows, 100000)
    r0 = rows // 3 if rows // 3 + pilot <= rows else 0
    t0 = time.perf_counter()
    ob.matvec_rows(bonds, x, r0, r0 + pilot)
    rate = pilot / max(time.perf_counter() - t0, 1e-6)
    n = int(min(rows, max(pilot, rate * 3.0)))
    r0 = min(r0, rows - n)
    nnz = ob.count_nnz(bonds, r0, r0 + n)
    for _ in range(args.warmup):
        ob.matvec_rows(bonds, x, r0, r0 + n)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        ob.matvec_rows(bonds, x, r0, r0 + n)
    dt = time.perf_counter() - t0
    val = nnz * args.steps / dt / 1e9
    sample = f"rows [{r0}, {r0 + n}) of {rows} per step ({nnz} nnz), FP64"
    out = {"impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": ws,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / args.steps * 1e3,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": {"workload": workload_name(inst, parity), "dim": rows, "n_sites": inst.n_sites,
                                          "two_s": inst.two_s, "two_m": inst.two_m, "l2": "inputs larger than L2"},
           "cpu_baseline": {"value": val, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))
    return 0


def oracle_free_uniform(seed, n):
    import numpy as np
    return np.random.default_rng(seed).uniform(-1.0, 1.0, n)


def run_grad(args):
    """Config 4: one step = y = H(J) x through the autograd function (HeisenbergMatvec), the
    loss L = g.y and its backward: dL/dx = H g and dL/dJ_b = -g^T (s_u.s_v) x.  Gnnz/s counts
    the three passes over the sector's nonzeros (forward product, backward product, bond
    correlations)."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_0706_3293_gb300 import api
    from paper_0706_3293_gb300.autograd import HeisenbergMatvec
    inst = instance(args.workload)
    dev = torch.device("cuda", torch.cuda.current_device())
    st = torch.cuda.current_stream()
    b = api.Basis(inst.n_sites, inst.two_s, inst.two_m)
    nnz = WORKLOADS[args.workload]
    xs, gs = oracle_free_uniform(inst.seed, b.dim), oracle_free_uniform(inst.seed + 1, b.dim)
    x0 = torch.from_numpy(xs).to(dev)
    g = torch.from_numpy(gs).to(dev)
    Jd = torch.from_numpy(inst.J.copy()).to(dev)

    def step(x, J):
        y = HeisenbergMatvec.apply(x, J, b, inst.u, inst.v)
        (g * y).sum().backward()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    x = x0.clone().requires_grad_(True)
    J = Jd.clone().requires_grad_(True)
    for _ in range(args.warmup):
        step(x, J)
        x.grad = None; J.grad = None
    barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    ev[0].record(st)
    for k in range(args.steps):
        y = HeisenbergMatvec.apply(x, J, b, inst.u, inst.v)
        ev[2 * k + 1].record(st)
        (g * y).sum().backward()
        ev[2 * k + 2].record(st)
        x.grad = None; J.grad = None
    barrier()
    clocks = sampler.stop() if sampler else None
    total_ms = ev[0].elapsed_time(ev[-1])
    fwd_ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    t_max = max_over_ranks(total_ms, ws, dev)
    value = 3 * nnz * args.steps * ws / (t_max * 1e-3) / 1e9
    # end to end: x and g from pinned host memory, both gradients back to the host, per step
    xh = torch.from_numpy(xs).pin_memory()
    gh = torch.from_numpy(gs).pin_memory()
    gxh = torch.empty(b.dim, dtype=torch.float64).pin_memory()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for k in range(args.steps):
        xd = xh.to(dev, non_blocking=True).requires_grad_(True)
        gd = gh.to(dev, non_blocking=True)
        Jk = Jd.clone().requires_grad_(True)
        y = HeisenbergMatvec.apply(xd, Jk, b, inst.u, inst.v)
        (gd * y).sum().backward()
        gxh.copy_(xd.grad, non_blocking=True)
        gJ = Jk.grad.cpu()
    e1.record(st)
    barrier()
    e2e_val = 3 * nnz * args.steps * ws / (max_over_ranks(e0.elapsed_time(e1), ws, dev) * 1e-3) / 1e9
    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    peak, peak_src = read_peaks()
    fwd_mean = float(np.mean(fwd_ms))
    achieved = ALGO_BYTES_PER_ROW * b.dim / (fwd_mean * 1e-3) / 1e9
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": inst.name + "_grad", "n_sites": inst.n_sites, "dim": b.dim,
                   "nnz_per_product": nnz, "products_per_step": 3, "bonds": inst.n_bonds,
                   "step": "autograd forward y = H x, backward dL/dx = H g and dL/dJ",
                   "parallelism": f"replicas{ws}", "l2": "inputs smaller than L2 (21.6 MB vectors)"},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": None,
                     "kernel": api.matvec_kernel_name(b, api.bonds_of(inst)) + " (forward)",
                     "peak_source": peak_src, "algorithmic_bytes_per_launch": ALGO_BYTES_PER_ROW * b.dim,
                     "mean_launch_ms": fwd_mean},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 2 * 8 * b.dim,
                "d2h_bytes_per_step": 8 * b.dim + 8 * inst.n_bonds},
        "gpu_launches": 4 * args.steps,
        "clocks": clocks,
        "grad_check": {"dL_dJ_first": float(gJ[0])},
    }
    if ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = grad_oracle_rate(inst, nnz, 1)
    print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def grad_oracle_rate(inst, nnz, reps):
    """The oracle's forward product, backward product and bond correlations on the whole
    sector, all host cores: (value, seconds per step, sample)."""
    import oracle
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bonds = oracle.Bonds(inst.u, inst.v, inst.J)
    xs, gs = oracle_free_uniform(inst.seed, ob.dim), oracle_free_uniform(inst.seed + 1, ob.dim)
    t0 = time.perf_counter()
    for _ in range(reps):
        ob.matvec(bonds, xs)
        ob.matvec(bonds, gs)
        ob.bond_corr(bonds, gs, xs)
    dt = (time.perf_counter() - t0) / reps
    return {"value": 3 * nnz / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the whole sector ({ob.dim} rows): forward and backward products and the "
                      f"bond correlations, {dt:.2f} s per step"}


def run_ftlm(args):
    """One step = one whole finite-temperature run: all 25 sectors of the N = 24 ring, 32
    +-1 vectors each, 80 Lanczos steps, in one graph launch through the C ABI.  Gnnz/s
    counts every executed vector-step: sum over (sector, vector) of nnz_A x Krylov length."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_0706_3293_gb300 import api
    inst = instance(args.workload)
    R = inst.meta["R"]
    bl = api.bonds_of(inst)
    temps = [0.25, 0.5, 1.0, 2.0, 4.0]
    for _ in range(args.warmup):
        res = api.ftlm_run(inst.n_sites, bl, R, inst.steps, inst.seed, temps)
    nnz_sec = [sector_nnz_s12(inst.n_sites, inst.n_bonds, A) for A in range(inst.n_sites + 1)]
    work = float(sum(nnz_sec[A] * int(res.mlen[A, :R].sum()) for A in range(inst.n_sites + 1)))
    st = torch.cuda.current_stream()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        res = api.ftlm_run(inst.n_sites, bl, R, inst.steps, inst.seed, temps)
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    if ws > 1 and rank != 0:
        import torch.distributed as dist
        dist.destroy_process_group()
        return 0
    value = work * args.steps * ws / (ms * 1e-3) / 1e9
    peak, peak_src = read_peaks()
    # algorithmic bytes of one Lanczos step on R FP32 vectors: product 8 B per vector-row
    # (read x, write u), update 12 B (read u and q, write w) = 20 B per vector-row
    rows = 2 ** inst.n_sites
    algo = 20.0 * rows * R * inst.steps
    achieved = algo / (ms / args.steps * 1e-3) / 1e9
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": inst.name, "n_sites": inst.n_sites, "sectors": inst.n_sites + 1,
                      "R": R, "lanczos_steps": inst.steps, "vector_nnz_per_run": work,
                      "vt": res.vt, "step": "one finite-temperature run (all sectors)",
                      "l2": "inputs larger than L2 (2 x %.1f GB vector sets)" % (rows * 32 * 4 / 1e9)},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": read_traffic("k_ftlm", inst.name),
                        "kernel": "k_ftlm (whole run)", "peak_source": peak_src,
                        "algorithmic_bytes_per_launch": algo},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 8 * inst.n_bonds * 2 + 8 * len(temps),
                   "d2h_bytes_per_step": 16 * len(temps) + 16 * 25 * 32 * inst.steps},
           "gpu_launches": 4 * args.steps, "clocks": clocks,
           "thermo": {"T": temps, "Z_rel": list(map(float, res.Z)), "E": list(map(float, res.E)),
                      "e_ref": res.e_ref}}
    print(json.dumps(out))
    return 0


def arnoldi_algo_bytes(dim: int, m: int) -> float:
    """Minimum bytes of an m-step Arnoldi run with classical Gram-Schmidt applied twice:
    per step the product (read v_j, write w: 16 B a row), per pass the dots (read the j
    basis vectors and w) and the update (read them again, read and write w), then |w| (read
    w) and v_{j+1} = w / |w| (read w, write v)."""
    tot = 0
    for j in range(1, m + 1):
        tot += 16 + 2 * 8 * (2 * j + 3) + 8 + 16
    return float(tot) * dim


def arnoldi_oracle_rate(inst, nnz, steps):
    """The oracle's Arnoldi (C products, numpy Gram-Schmidt) on the first `steps` steps of
    the same run, all host cores: products' nnz per second."""
    import oracle
    ob = oracle.Basis(inst.n_sites, inst.two_s, inst.A)
    bonds = oracle.Bonds(inst.u, inst.v, inst.J)
    v0 = oracle.start_uniform(inst.seed, ob.dim)
    t0 = time.perf_counter()
    _, m = oracle.arnoldi(ob, bonds, v0, steps)
    dt = time.perf_counter() - t0
    return {"value": nnz * m / dt / 1e9, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
            "sample": f"the first {m} of the {inst.steps} Arnoldi steps ({dt:.1f} s)"}, dt


def run_arnoldi(args):
    """One step = one whole Arnoldi run (60 steps, full re-orthogonalisation) through the C
    ABI (arnoldi_run): products and Gram-Schmidt kernels, Ritz values on the host."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_0706_3293_gb300 import api
    inst = instance(args.workload)
    b = api.Basis(inst.n_sites, inst.two_s, inst.two_m)
    bl = api.bonds_of(inst)
    nnz = WORKLOADS[args.workload]
    for _ in range(args.warmup):
        res = api.arnoldi_run(b, bl, inst.steps, seed=inst.seed, n_ritz=3)
    m = res.steps
    st = torch.cuda.current_stream()
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(args.steps):
        res = api.arnoldi_run(b, bl, inst.steps, seed=inst.seed, n_ritz=3)
    e1.record(st)
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    # end to end: the start vector from pinned host memory, H and the Ritz values back
    x_host = torch.empty(b.dim, dtype=torch.float64, pin_memory=True)
    x_host.copy_(api.start_vector(b, inst.seed, dtype=torch.float64).cpu())
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        v0 = x_host.to("cuda", non_blocking=True)
        res2 = api.arnoldi_run(b, bl, inst.steps, v0=v0, n_ritz=3)
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1), ws, "cuda")
    if ws > 1 and rank != 0:
        import torch.distributed as dist
        dist.destroy_process_group()
        return 0
    value = nnz * m * args.steps * ws / (ms * 1e-3) / 1e9
    peak, peak_src = read_peaks()
    algo = arnoldi_algo_bytes(b.dim, m)
    achieved = algo / (ms / args.steps * 1e-3) / 1e9
    # launches per run: start (seeded vector, norm, start, scale), per step the product
    # (exponent pre-pass + block kernel), 2 x (dots, their sums, update), norm, beta, scale
    launches = 4 + m * (2 + 2 * 3 + 3)
    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": inst.name, "n_sites": inst.n_sites, "dim": b.dim, "arnoldi_steps": m,
                      "nnz_per_product": nnz, "step": "one whole Arnoldi run",
                      "l2": "inputs larger than L2 (%d basis vectors of %.1f MB)" % (m + 1, b.dim * 8 / 1e6)},
           "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                        "frac": achieved / peak, "traffic": None,
                        "kernel": "arnoldi_run (all kernels of the run)", "peak_source": peak_src,
                        "algorithmic_bytes_per_launch": algo},
           "e2e": {"value": nnz * m * args.steps * ws / (e2e_ms * 1e-3) / 1e9, "unit": UNIT,
                   "h2d_bytes_per_step": 8 * b.dim, "d2h_bytes_per_step": 8 * (inst.steps + 1) * inst.steps + 24},
           "gpu_launches": launches * args.steps, "clocks": clocks,
           "ritz": list(map(float, res.ritz))}
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"], _ = arnoldi_oracle_rate(inst, nnz, 6)
    print(json.dumps(out))
    return 0


def launches_per_step(kname: str, dtype: str, momentum) -> int:
    """Kernels one Lanczos step launches: product (+ second pass of the split product) and
    the alpha reduction; update and beta reduction; on the FP64 block paths the fixed-point
    copy of the new vector; on a momentum basis the product's separate epilogue."""
    n = 4
    if "+" in kname:
        n += 1
    if dtype == "f64" and ("blk_lz64" in kname or "s1_lz64" in kname):
        n += 1
    if momentum is not None:
        n += 1
    return n


def splitmix64(seed: int, t: int) -> int:
    """Output t of SplitMix64 (Steele, Lea, Flood 2014) seeded with seed: the key of a
    finite-temperature start vector (sector A, vector r) is output A 2^20 + r of the run's
    seed."""
    M = (1 << 64) - 1
    z = (seed + (t + 1) * 0x9E3779B97F4A7C15) & M
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M
    return z ^ (z >> 31)


def compare_forms(api, torch, b, bl, inst, nnz, steps=150):
    """The FP32 and batched forms against the plain FP64 form on this GPU, each at the
    ground energy it reaches.  FP64 and FP32: whole Lanczos runs (one graph each) of `steps`
    steps on the default sector, the lowest Ritz value against the Majumdar-Ghosh energy
    -3N/8 (J2 = J1/2) and against each other.  Batched: one finite-temperature run of the
    N = 24 ring (all sectors, 32 vectors, 80 steps), its M = 0 vector r = 0 against a plain
    FP64 run of 80 steps from the same +-1 vector, and that plain FP64 form's rate on the
    same sector."""
    import numpy as np
    st = torch.cuda.current_stream()

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(st)
        r = fn()
        e1.record(st)
        torch.cuda.synchronize()
        return r, e0.elapsed_time(e1)

    out = {}
    e_mg = -3.0 * inst.n_sites / 8.0
    res = {}
    for dt, tdt in (("f64", torch.float64), ("f32", torch.float32)):
        ws = torch.empty(api.lanczos_workspace(b, tdt, steps), dtype=torch.uint8, device="cuda")
        api.lanczos_run(b, bl, 3, seed=inst.seed, dtype=tdt, n_ritz=1, work=ws)   # warm-up
        r, ms = timed(lambda: api.lanczos_run(b, bl, steps, seed=inst.seed, dtype=tdt, n_ritz=1, work=ws))
        del ws
        torch.cuda.empty_cache()
        res[dt] = (r, ms)
        out[dt] = {"workload": inst.name, "steps": int(r.steps_done), "ms_per_step": ms / r.steps_done,
                   "gnnz_s": nnz * r.steps_done / (ms * 1e-3) / 1e9, "E0": float(r.ritz[0]),
                   "rel_err_vs_exact": abs(float(r.ritz[0]) - e_mg) / abs(e_mg),
                   "exact": f"Majumdar-Ghosh -3N/8 = {e_mg}"}
    out["f32"]["rel_err_vs_f64"] = abs(out["f32"]["E0"] - out["f64"]["E0"]) / abs(out["f64"]["E0"])
    out["f32"]["speedup_vs_f64"] = out["f32"]["gnnz_s"] / out["f64"]["gnnz_s"]
    # batched finite-temperature run
    fi = instance("ftlm_ring24")
    R = fi.meta["R"]
    fb = api.bonds_of(fi)
    api.ftlm_run(fi.n_sites, fb, R, fi.steps, fi.seed, [1.0])                      # warm-up, tiling
    fr, fms = timed(lambda: api.ftlm_run(fi.n_sites, fb, R, fi.steps, fi.seed, [1.0]))
    nnz_sec = [sector_nnz_s12(fi.n_sites, fi.n_bonds, A) for A in range(fi.n_sites + 1)]
    vsteps = int(fr.mlen[:, :R].sum())
    work = float(sum(nnz_sec[A] * int(fr.mlen[A, :R].sum()) for A in range(fi.n_sites + 1)))
    A0 = fi.n_sites // 2
    b24 = api.Basis(fi.n_sites, 1, 0)
    v0 = api.start_vector(b24, splitmix64(fi.seed, (A0 << 20) + 0), kind=1, dtype=torch.float64)
    api.lanczos_run(b24, fb, 3, v0=v0, n_ritz=1)
    r64, ms64 = timed(lambda: api.lanczos_run(b24, fb, fi.steps, v0=v0, n_ritz=1))
    m = int(fr.mlen[A0, 0])
    e32 = float(np.min(fr.theta[A0, 0, :m]))
    g_plain = nnz_sec[A0] * r64.steps_done / (ms64 * 1e-3) / 1e9
    g_batch = work / (fms * 1e-3) / 1e9
    out["batched"] = {"workload": fi.name, "sectors": fi.n_sites + 1, "R": R, "steps": fi.steps,
                      "ms_per_run": fms, "vector_steps": vsteps, "ms_per_vector_step": fms / vsteps,
                      "gnnz_s": g_batch, "E0_M0_r0": e32, "E0_M0_r0_f64": float(r64.ritz[0]),
                      "rel_err_vs_f64": abs(e32 - float(r64.ritz[0])) / abs(float(r64.ritz[0])),
                      "f64_same_sector": {"ms_per_step": ms64 / r64.steps_done, "gnnz_s": g_plain},
                      "speedup_vs_f64_same_sector": g_batch / g_plain,
                      "speedup_vs_f64_default": g_batch / out["f64"]["gnnz_s"]}
    b24.close()
    return out


def run_ours(args):
    if args.workload == "arnoldi_ring24":
        return run_arnoldi(args)
    if args.workload == "ring24_grad":
        return run_grad(args)
    if args.workload == "ftlm_ring24":
        return run_ftlm(args)
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    import __graft_entry__
    __graft_entry__.build()
    from paper_0706_3293_gb300 import api

    inst = instance(args.workload)
    dtype = args.dtype or DEFAULT_DTYPE.get(args.workload, "f64")
    tdt = torch.float64 if dtype == "f64" else torch.float32
    dev = torch.device("cuda", torch.cuda.current_device())
    parity = PARITY.get(args.workload, 0)
    momentum = MOMENTUM.get(args.workload)
    b = api.Basis(inst.n_sites, inst.two_s, inst.two_m, parity=parity, momentum=momentum)
    bl = api.bonds_of(inst)
    nnz = WORKLOADS[args.workload] or api.count_nnz(b, bl)
    total = args.warmup + args.steps
    st = torch.cuda.current_stream()

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    # ---- device-resident timing ----
    run = api.LanczosRun(b, bl, total, seed=inst.seed, dtype=tdt)
    kname = run.kernel_name()
    for _ in range(args.warmup):
        run.step()
    barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    if sampler:
        sampler.start()
        time.sleep(0.4)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
    ev[0].record(st)
    for k in range(args.steps):
        run.substep(0)
        ev[2 * k + 1].record(st)
        run.substep(1)
        ev[2 * k + 2].record(st)
    barrier()
    clocks = sampler.stop() if sampler else None
    total_ms = ev[0].elapsed_time(ev[-1])
    mv_ms = [ev[2 * k].elapsed_time(ev[2 * k + 1]) for k in range(args.steps)]
    al, be, rc = run.read()
    run.close()
    del run
    t_max = max_over_ranks(total_ms, ws, dev)
    value = nnz * args.steps * ws / (t_max * 1e-3) / 1e9

    # ---- end to end through the C ABI with host buffers ----
    x_host = torch.empty(b.dim, dtype=tdt, pin_memory=True)
    x_host.copy_(api.start_vector(b, inst.seed, dtype=tdt).cpu())
    torch.cuda.synchronize()
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(st)
    v0 = x_host.to(dev, non_blocking=True)
    run2 = api.LanczosRun(b, bl, args.steps, v0=v0, dtype=tdt)
    d2h = 0
    for k in range(args.steps):
        run2.step()
        a2, b2, _ = run2.read()      # the step's result (alpha_j, beta_j) back on the host
        d2h += 16
    e1.record(st)
    barrier()
    e2e_ms = e0.elapsed_time(e1)
    run2.close()
    del run2, v0
    e2e_val = nnz * args.steps * ws / (max_over_ranks(e2e_ms, ws, dev) * 1e-3) / 1e9

    if rank != 0:
        if ws > 1:
            import torch.distributed as dist
            dist.destroy_process_group()
        return 0
    peak, peak_src = read_peaks()
    mv_mean = float(np.mean(mv_ms))
    algo_row = ALGO_BYTES_PER_ROW if dtype == "f64" else ALGO_BYTES_PER_ROW // 2
    achieved = algo_row * b.dim / (mv_mean * 1e-3) / 1e9
    traffic = read_traffic(kname, workload_name(inst, parity, momentum))
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic",
        "config": {"workload": workload_name(inst, parity, momentum), "n_sites": inst.n_sites, "two_s": inst.two_s,
                   "two_m": inst.two_m, "dim": b.dim, "nnz_per_product": nnz,
                   "bonds": inst.n_bonds, "start_seed": inst.seed, "parallelism": f"replicas{ws}",
                   "l2": "inputs larger than L2 (2 x %.1f GB vectors)" % (b.dim * 8 / 1e9)},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": kname, "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": algo_row * b.dim,
                     "mean_launch_ms": mv_mean},
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": b.dim * (8 if dtype == "f64" else 4) / args.steps,
                "d2h_bytes_per_step": 16},
        # per step: the product (two passes when split), alpha, update, beta, and on the FP64
        # block paths the fixed-point copy; on a momentum basis the product's epilogue
        "gpu_launches": launches_per_step(kname, dtype, momentum) * args.steps,
        "clocks": clocks,
        "lanczos": {"alpha_last": float(al[-1]) if len(al) else None,
                    "steps_done": int(len(al)), "status": int(rc)},
    }
    if ws == 1 and not args.no_compare and args.workload == "j1j2_ring32" and dtype == "f64":
        out["forms"] = compare_forms(api, torch, b, bl, inst, nnz)
    if ws == 1 and not args.no_cpu_baseline and momentum is None:
        out["cpu_baseline"] = cpu_baseline(inst, nnz, parity=parity)
    elif ws == 1 and not args.no_cpu_baseline:
        out["cpu_baseline"] = {"value": None, "unit": UNIT, "cores": 0, "kind": "oracle",
                               "sample": "none: the oracle builds momentum blocks densely, for small N only"}
    print(json.dumps(out))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="j1j2_ring32", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip the FP32 and batched comparison runs of the default workload")
    ap.add_argument("--dtype", choices=["f64", "f32"], default=None,
                    help="Lanczos vector type (default: f64; f32 for s1_rrg20)")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
