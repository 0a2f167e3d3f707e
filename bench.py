#!/usr/bin/env python
"""Benchmark of the TreeCode hot path on GB300.

One step = one kick-drift-kick leapfrog step (Eqs. 2-5) of the whole hot
path: kick+drift+box, Morton keys, onesweep sort, octree, gather, FP64
moments, FP32 tree walk with the fused force write-back and final kick, and
the FP64 diagnostics reductions.  Workload: the galaxy-like model at
N = 1e8 (exponential disk 60 %, Hernquist bulge 10 %, truncated NFW-like
halo 30 %), eps = 0.02, theta = 0.7, quadrupole cells, leaf <= 16, groups of
32, tau = 0.002, FP32 with Kahan-compensated sums.  Inputs are seeded
synthetic particles, resident in HBM, 4+ GB (far larger than L2).

Prints one JSON line.  --impl reference times the FP64 CPU oracle on the
host cores instead (a bounded sample of the same workload).
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "tree-force particles/s at N=1e8 θ=0.7, FP32 vs FP64 GPU at force err ≤1e-3"
UNIT = "particles/s"
SEED = 20241202
PARAMS = dict(eps=0.02, theta=0.7, order=2, leaf_cap=16, group_size=32, kahan=1)
TAU = 0.002
WORKLOAD = ("galaxy-like N=1e8: exp. disk 60% (R_d=1, z0=0.1) + Hernquist bulge 10% (a=0.2) + "
            "NFW-like halo 30% (r_s=5, r_t=50), eps=0.02, theta=0.7, quadrupole, leaf<=16, "
            "KDK tau=0.002")
# Algorithmic flop counts per pair (FMA = 2 flops; rsqrt = 1): PP with
# potential 20, PC quadrupole 54, PC monopole 20.
FLOPS_PP, FLOPS_PC_QUAD, FLOPS_PC_MONO = 20, 54, 20
# FP32 peak derived from unit counts and clocks: 152 SMs x 128 FP32 lanes x
# 2 flops (FMA) x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DRAM bytes per walk launch from ncu (dram__bytes_read.sum + write.sum) on the
# N = 1e7 galaxy case of the same kernel, per particle (scaled by N below);
# None when the kernel has changed since the counters were taken.
WALK_DRAM_BYTES_PER_PARTICLE = 1010


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=float, default=1e8)
    ap.add_argument("--cpu-sample", type=int, default=1 << 20,
                    help="particles of the oracle's bounded sample (same galaxy recipe)")
    ap.add_argument("--no-extras", action="store_true",
                    help="time the main leg only (no FP64 leg, error check, e2e, CPU baseline)")
    ap.add_argument("--study", choices=["theta", "threads", "ensemble", "adjoint", "plain"], default=None,
                    help="theta: precision study on the Plummer N=2^20 config (force error vs direct sum, "
                         "energy drift, FP32 vs FP64 time per force, theta in {0.4,0.5,0.7,1.0}); "
                         "threads: T(M), speedup and efficiency of the CPU oracle vs host threads M; "
                         "ensemble: 512 Plummer clusters in one build, autotuned, one CUDA graph per step; "
                         "adjoint: gradients through 16 KDK steps of Plummer N=262144 (times, FP32 vs FP64, "
                         "tree vs theta=0, finite differences); plain: the FP64 Plummer N=16384 configuration "
                         "(tree vs direct error, 10 KDK steps, energy and momentum drift, GPU vs oracle)")
    ap.add_argument("--study-steps", type=int, default=100)
    ap.add_argument("--err-samples", type=int, default=100000,
                    help="particles whose tree force is checked against the GPU direct sum (extras)")
    ap.add_argument("--nvtx", action="store_true",
                    help="mark each timed step with an NVTX range named 'step' (for profiler selection)")
    return ap.parse_args()


# ----------------------------------------------------------------- clocks
class Clocks:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([c.strip() for c in line.split(",")])

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in self.rows:
            try:
                sm.append(float(r[1])); mx.append(float(r[2]))
                for nm, val in zip(names, r[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------- ranks
# One process per GPU.  The galaxy step is one problem, so N ranks run N
# independent replicas (seed + rank); an ensemble is split by system with no
# exchange at all.  Timing is the maximum over ranks.
def max_over_ranks(v, world, device):
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def rank_share(sizes, rank, world):
    """Systems of an ensemble owned by `rank`: largest first, each to the least
    loaded rank (ties to the lower rank), so particle counts stay balanced."""
    load = [0] * world
    own = [[] for _ in range(world)]
    for b in sorted(range(len(sizes)), key=lambda b: (-int(sizes[b]), b)):
        r = min(range(world), key=lambda q: (load[q], q))
        own[r].append(b)
        load[r] += int(sizes[b])
    return sorted(own[rank])


# ----------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    import torch.distributed as dist

    from paper_2412_01733_gb300 import build, inputs, treegb

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    build.build()
    n = int(a.n)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    # each rank runs its own replica of the workload (independent seeds)
    x, v, m = inputs.galaxy(n, SEED + rank, device=dev, dtype=torch.float32)
    x, v, m = x.contiguous(), v.contiguous(), m.contiguous()
    ws = treegb.Workspace(n, **PARAMS)
    acc, phi = ws.accel(x, m)
    diag = torch.empty(8, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()

    def step():
        ws.leapfrog_step(x, v, m, acc, TAU, phi=phi)
        ws.diagnostics(x, v, m, phi, out=diag)

    for _ in range(a.warmup):
        step()
    torch.cuda.synchronize()
    if ws.status() != 0:
        raise RuntimeError("device status set during warm-up")
    d0 = diag.cpu().numpy().copy()

    clocks = Clocks(local)
    barrier()
    torch.cuda.synchronize()
    ws.timing(True)
    clocks.start()
    evs = [torch.cuda.Event(enable_timing=True) for _ in range(a.steps + 1)]
    e0, e1 = evs[0], evs[-1]
    e0.record(stream)
    for k in range(a.steps):
        if a.nvtx:
            torch.cuda.nvtx.range_push("step")
        step()
        if a.nvtx:
            torch.cuda.nvtx.range_pop()
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    per_step = [evs[k].elapsed_time(evs[k + 1]) for k in range(a.steps)]
    barrier()
    ck = clocks.stop()
    t = max_over_ranks(e0.elapsed_time(e1) / 1e3, world, dev)
    phases, launches = ws.timing_read()
    ws.timing(False)
    inf = ws.info()
    st = ws.status()
    if st != 0:
        raise RuntimeError(f"device status {st} in the timed region")
    d1 = diag.cpu().numpy().copy()
    value = world * n * a.steps / t

    # roofline of the dominant kernel: the FP32 walk
    walk_ms, walk_calls = phases["walk"]
    walk_s = walk_ms / 1e3 / max(walk_calls, 1)
    flops = FLOPS_PP * inf["pp_pairs"] + FLOPS_PC_QUAD * inf["pc_pairs"]
    achieved = flops / walk_s / 1e12
    traffic = None if WALK_DRAM_BYTES_PER_PARTICLE is None else WALK_DRAM_BYTES_PER_PARTICLE * n
    roofline = {"bound": "alu", "kernel": "k_walk<float,1,quad,kahan,soft,force>", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": traffic,
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 x 2.07 GHz (no FP32 entry in MEASURED_PEAKS)",
                "flops_per_launch": flops, "pp_pairs": inf["pp_pairs"], "pc_pairs": inf["pc_pairs"],
                "walk_ms": walk_s * 1e3}
    step_ms = t * 1e3 / a.steps
    sem = statistics.stdev(per_step) / math.sqrt(len(per_step)) if len(per_step) > 1 else None
    breakdown = {k: round(ms / a.steps, 3) for k, (ms, c) in phases.items() if c}

    out = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": step_ms, "ms_per_step_sem": sem, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": n, "group_size": PARAMS["group_size"],
                      "leaf_cap": PARAMS["leaf_cap"], "kahan": True, "parallelism": f"replicas{world}",
                      "l2": "inputs (4+ GB) larger than L2 (129 MB)"},
           "gpu_launches": launches, "roofline": roofline, "phase_ms_per_step": breakdown,
           "interactions_per_s": world * (inf["pp_pairs"] + inf["pc_pairs"]) / walk_s,
           "interactions_per_particle": (inf["pp_pairs"] + inf["pc_pairs"]) / n,
           "tree": {"nodes": inf["n_nodes"], "depth": inf["depth"], "max_stack": inf["max_stack"]},
           "energy_rel_drift": float(abs((d1[0] + d1[1]) - (d0[0] + d0[1])) / abs(d0[0] + d0[1])),
           "clocks": ck}

    if not a.no_extras:
        # end to end through the C ABI with host-resident state (first among the extras,
        # right after the timed steps)
        xh = x.cpu().pin_memory(); vh = v.cpu().pin_memory(); mh = m.cpu().pin_memory()
        ah = acc.cpu().pin_memory(); dh = torch.empty(8, dtype=torch.float64).pin_memory()

        part_ev = []

        def e2e_step():
            ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            ev[0].record(stream)
            x.copy_(xh, non_blocking=True); v.copy_(vh, non_blocking=True)
            m.copy_(mh, non_blocking=True); acc.copy_(ah, non_blocking=True)
            ev[1].record(stream)
            ws.leapfrog_step(x, v, m, acc, TAU, phi=phi)
            ws.diagnostics(x, v, m, phi, out=diag)
            ev[2].record(stream)
            xh.copy_(x, non_blocking=True); vh.copy_(v, non_blocking=True)
            ah.copy_(acc, non_blocking=True); dh.copy_(diag, non_blocking=True)
            ev[3].record(stream)
            part_ev.append(ev)

        e2e_step()
        torch.cuda.synchronize()
        barrier()
        clocks_e2e = Clocks(local)
        clocks_e2e.start()
        h0 = torch.cuda.Event(enable_timing=True); h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(a.steps):
            e2e_step()
        h1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck_e2e = clocks_e2e.stop()
        te = max_over_ranks(h0.elapsed_time(h1) / 1e3, world, dev)
        timed_ev = part_ev[-a.steps:]
        split = {k: sum(ev[i].elapsed_time(ev[i + 1]) for ev in timed_ev) / a.steps
                 for i, k in enumerate(("h2d_ms", "step_ms", "d2h_ms"))}
        out["e2e"] = {"value": world * n * a.steps / te, "unit": UNIT,
                      "h2d_bytes_per_step": 40 * n, "d2h_bytes_per_step": 36 * n + 64, "clocks": ck_e2e,
                      "per_step": {k: round(v, 2) for k, v in split.items()}}
        del xh, vh, mh, ah, dh
        # force error of the FP32 tree against the GPU direct sum (sampled particles; the state
        # after the end-to-end steps, whose accelerations belong to these positions)
        g = torch.Generator().manual_seed(SEED)
        tgt = torch.randint(0, n, (min(n, a.err_samples),), generator=g)
        ad, _ = ws.direct(x, m, tgt, precision="f32")
        at = acc[:, tgt.to(dev)].double()
        err = ((at - ad).norm(dim=0) / ad.norm(dim=0)).cpu()
        out["force_err_vs_direct"] = {"median": float(err.median()), "p99": float(err.quantile(0.99)),
                                      "max": float(err.max()), "samples": int(tgt.numel()),
                                      "reference": "GPU direct sum, FP32 pairs, compensated, FP64 chunk totals"}
        # same-GPU FP64 plain path: one force evaluation (build + moments + walk) on the same state
        x64, m64 = x.double().contiguous(), m.double().contiguous()
        del ad
        torch.cuda.synchronize()
        ws64 = treegb.Workspace(n, precision="f64", **{k: v for k, v in PARAMS.items() if k != "kahan"})
        ws64.accel(x64, m64)
        ws64.timing(True)
        f0 = torch.cuda.Event(enable_timing=True); f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        a64, p64 = ws64.accel(x64, m64)
        f1.record(stream)
        torch.cuda.synchronize()
        ph64, _ = ws64.timing_read()
        t64 = f0.elapsed_time(f1) / 1e3
        ws.timing(True)
        g0 = torch.cuda.Event(enable_timing=True); g1 = torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        a32, p32 = ws.accel(x, m)
        g1.record(stream)
        torch.cuda.synchronize()
        ph32, _ = ws.timing_read()
        ws.timing(False)
        t32 = g0.elapsed_time(g1) / 1e3
        e64 = ((a32.double()[:, tgt.to(dev)] - a64[:, tgt.to(dev)]).norm(dim=0)
               / a64[:, tgt.to(dev)].norm(dim=0)).cpu()
        out["fp32_vs_fp64"] = {"fp32_force_particles_per_s": n / t32, "fp64_force_particles_per_s": n / t64,
                               "speedup": t64 / t32, "fp32_walk_ms": ph32["walk"][0],
                               "fp64_walk_ms": ph64["walk"][0],
                               "fp32_vs_fp64_median_rel": float(e64.median()),
                               "fp32_vs_fp64_max_rel": float(e64.max())}
        del ws64, x64, m64, a64, p64, a32, p32
        torch.cuda.synchronize()
        torch.cuda.empty_cache()
        # the FP64 CPU oracle on the host cores, bounded sample, rank 0 at N = 1 only
        if world == 1:
            out["cpu_baseline"] = cpu_baseline(a.cpu_sample)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def cpu_baseline(ns):
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2412_01733_gb300 import inputs
    x, _, m = inputs.galaxy(ns, SEED, dtype=torch.float64)
    x, m = x.numpy(), m.numpy()
    t0 = time.perf_counter()
    O.tree_forces(x, m, eps=PARAMS["eps"], theta=PARAMS["theta"], lcap=PARAMS["leaf_cap"],
                  gs=PARAMS["group_size"], quad=True)
    t = time.perf_counter() - t0
    return {"value": ns / t, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
            "sample": f"one FP64 tree-force evaluation (box, keys, sort, octree, moments, lists, forces) "
                      f"of the same galaxy recipe at N={ns} (not 1e8); {t:.2f} s"}


# ----------------------------------------------------------------- reference arm (the oracle)
def run_reference(a):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2412_01733_gb300 import inputs
    ns = a.cpu_sample
    x, v, m = inputs.galaxy(ns, SEED, dtype=torch.float64)
    x, v, m = x.numpy(), v.numpy(), m.numpy()
    acc = lambda xx: O.tree_accel(xx, m, eps=PARAMS["eps"], theta=PARAMS["theta"], lcap=PARAMS["leaf_cap"],
                                  gs=PARAMS["group_size"], quad=True)
    st = acc(x)
    for _ in range(a.warmup):
        x, v, aa, ph = O.kdk(x, v, m, TAU, 1, acc, a0=st)
        st = (aa, ph)
    t0 = time.perf_counter()
    for _ in range(a.steps):
        x, v, aa, ph = O.kdk(x, v, m, TAU, 1, acc, a0=st)
        st = (aa, ph)
    t = time.perf_counter() - t0
    value = ns * a.steps / t
    sample = (f"FP64 CPU oracle KDK steps (tree rebuilt each step) of the same galaxy recipe at N={ns} "
              f"(bounded sample of the N=1e8 workload)")
    out = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": a.gpus,
           "steps": a.steps, "warmup": a.warmup, "ms_per_step": t * 1e3 / a.steps, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": WORKLOAD, "n": ns, "parallelism": "host threads"},
           "cpu_baseline": {"value": value, "unit": UNIT, "cores": O.threads(), "kind": "oracle",
                            "sample": sample},
           "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


# ----------------------------------------------------------------- studies
def study_theta(a):
    """Plummer N = 1,048,576, eps = 0.005, quadrupole cells, theta in {0.4, 0.5, 0.7, 1.0}: force error of
    the FP32 and FP64 tree against the FP64 direct sum on 4096 sampled particles, FP32 / FP64 time per
    force evaluation, and the relative energy drift over K KDK steps (tau = 0.005)."""
    import torch

    from paper_2412_01733_gb300 import build, inputs, treegb
    build.build()
    n, eps, tau = 1 << 20, 0.005, 0.005
    x, v, m = inputs.plummer(n, SEED, device="cuda", dtype=torch.float64)
    g = torch.Generator().manual_seed(SEED)
    tgt = torch.randint(0, n, (4096,), generator=g).cuda()
    ref_ws = treegb.Workspace(n, precision="f64", eps=eps)
    a_ref, p_ref = ref_ws.direct(x.contiguous(), m.contiguous(), tgt, precision="f64")
    del ref_ws

    def timed(fn):
        fn()
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        e0.record(); out = fn(); e1.record(); torch.cuda.synchronize()
        return out, e0.elapsed_time(e1)

    for theta in (0.4, 0.5, 0.7, 1.0):
        row = {"study": "theta", "n": n, "eps": eps, "theta": theta, "order": "quadrupole", "leaf_cap": 16}
        for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
            # explicit copies: the leapfrog below advances them in place
            xs, vs, ms = x.to(dt).clone(), v.to(dt).clone(), m.to(dt).clone()
            ws = treegb.Workspace(n, precision=prec, eps=eps, theta=theta)
            (acc, phi), ms_force = timed(lambda: ws.accel(xs, ms))
            e = ((acc[:, tgt].double() - a_ref).norm(dim=0) / a_ref.norm(dim=0)).cpu()
            inf = ws.info()
            row[prec] = {"force_ms": ms_force, "particles_per_s": n / (ms_force / 1e3),
                         "err_median": float(e.median()), "err_p99": float(e.quantile(0.99)),
                         "err_max": float(e.max()), "interactions_per_particle": (inf["pp_pairs"] + inf["pc_pairs"]) / n}
            steps = a.study_steps if prec == "f32" else max(1, a.study_steps // 10)
            d = ws.diagnostics(xs, vs, ms, phi).cpu().numpy()
            e0_ = d[0] + d[1]
            for _ in range(steps):
                ws.leapfrog_step(xs, vs, ms, acc, tau, phi=phi)
            d = ws.diagnostics(xs, vs, ms, phi).cpu().numpy()
            row[prec]["energy_drift"] = float(abs(d[0] + d[1] - e0_) / abs(e0_))
            row[prec]["drift_steps"] = steps
            if ws.status() != 0:
                row[prec]["status"] = ws.status()
            del ws, xs, vs, ms, acc, phi
            torch.cuda.empty_cache()
        row["fp32_speedup_vs_fp64"] = row["f64"]["force_ms"] / row["f32"]["force_ms"]
        print(json.dumps(row), flush=True)


def study_threads(a):
    """The paper's own measurement (Sec. 3, Eqs. 6-7) on the FP64 CPU oracle: mean time T(M) of one tree
    force evaluation over 10 repetitions with its standard error, speedup S = T(1)/T(M) and efficiency
    E = S/M, for M host threads, galaxy recipe at N = 1e5 and 1e6, theta = 1."""
    import os as _os

    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2412_01733_gb300 import inputs
    ncpu = _os.cpu_count() or 1
    ms_list = sorted({1, 2, 4, 8, ncpu // 2, ncpu} - {0})
    for n in (100_000, 1_000_000):
        x, _, m = inputs.galaxy(n, SEED, dtype=torch.float64)
        x, m = x.numpy(), m.numpy()
        res = {}
        for M in ms_list:
            O.set_threads(M)
            reps = 10 if n <= 100_000 else 5
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                O.tree_forces(x, m, eps=PARAMS["eps"], theta=1.0, lcap=PARAMS["leaf_cap"], gs=PARAMS["group_size"])
                ts.append(time.perf_counter() - t0)
            ts = np.array(ts)
            res[M] = (ts.mean(), ts.std(ddof=1) / np.sqrt(len(ts)))
        T1, dT1 = res[1]
        for M, (T, dT) in res.items():
            S = T1 / T
            dS = (T1 * dT + T * dT1) / (T * T)
            print(json.dumps({"study": "threads", "n": n, "threads": M, "host_cpus": ncpu, "T_s": T, "T_sem": dT,
                              "S": S, "S_err": dS, "E": S / M, "E_err": dS / M}), flush=True)
        O.set_threads(ncpu)
    # the direct sum of Eq. 1 (the paper's PP tool), N = 2^15, one thread and all
    x, _, m = inputs.galaxy(1 << 15, SEED, dtype=torch.float64)
    x, m = x.numpy(), m.numpy()
    for M in (1, ncpu):
        O.set_threads(M)
        t0 = time.perf_counter()
        O.direct(x, m, eps=PARAMS["eps"])
        print(json.dumps({"study": "threads_direct", "n": 1 << 15, "threads": M, "T_s": time.perf_counter() - t0}),
              flush=True)
    # efficiency against N at M = 4 threads (the paper's E(N) view), N = 2^17 .. 2^21
    for lg in range(17, 22):
        n = 1 << lg
        x, _, m = inputs.galaxy(n, SEED, dtype=torch.float64)
        x, m = x.numpy(), m.numpy()
        T = {}
        for M in (1, 4):
            O.set_threads(M)
            ts = []
            for _ in range(2):
                t0 = time.perf_counter()
                O.tree_forces(x, m, eps=PARAMS["eps"], theta=1.0, lcap=PARAMS["leaf_cap"], gs=PARAMS["group_size"])
                ts.append(time.perf_counter() - t0)
            T[M] = min(ts)
        print(json.dumps({"study": "threads_vs_n", "n": n, "threads": 4, "T1_s": T[1], "T4_s": T[4],
                          "S": T[1] / T[4], "E": T[1] / T[4] / 4}), flush=True)
    O.set_threads(ncpu)


def study_ensemble(a):
    """Ensemble configuration: 512 independent Plummer clusters (a = 1, M = 1 each), sizes
    N_c = floor(exp U(ln 1024, ln 65536)) (about 7.9e6 particles in all), eps = 0.01, theta = 0.6,
    quadrupole, FP32 + Kahan, KDK tau = 0.005.  The autotuner picks (leaf_cap, group_size,
    stack_depth); each step is then one CUDA graph launch (leapfrog step + diagnostics).  Reports
    particles/s and interactions/s of the step, the same steps launched eagerly, and the per-cluster
    relative energy drift over all steps run (median, max)."""
    import numpy as np
    import torch

    import torch.distributed as dist

    from paper_2412_01733_gb300 import build, inputs, treegb
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    B, tau = 512, 0.005
    x, v, m, off = inputs.ensemble(B, SEED, device=dev, dtype=torch.float32)
    n_all = x.shape[1]
    if world > 1:
        # this rank's systems (no exchange between ranks)
        own = rank_share(np.diff(off), rank, world)
        idx = torch.cat([torch.arange(int(off[b]), int(off[b + 1]), device=dev) for b in own])
        x, v, m = x[:, idx], v[:, idx], m[idx]
        off = np.concatenate(([0], np.cumsum(np.diff(off)[own]))).astype(np.int64)
        B = len(own)
    x, v, m = x.contiguous(), v.contiguous(), m.contiguous()
    n = x.shape[1]
    base = dict(eps=0.01, theta=0.6, order=2, kahan=1, leaf_cap=16, group_size=32)
    t0 = time.perf_counter()
    best, table = treegb.autotune(x, m, offsets=off, reps=3, **base)
    tune_s = time.perf_counter() - t0
    p = dict(base, leaf_cap=best.leaf_cap, group_size=best.group_size, stack_depth=best.stack_depth)
    ws = treegb.Workspace(n, **p)
    ws.set_segments(off)
    acc, phi = ws.accel(x, m)
    d0 = ws.diagnostics_segments(x, v, m, phi).cpu().numpy()
    diag = torch.zeros(8, dtype=torch.float64, device="cuda")
    ws.graph_capture(x, v, m, acc, tau, phi=phi, diag=diag)
    s = torch.cuda.current_stream()

    def timed(fn, k):
        e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(); e0.record(s)
        for _ in range(k):
            fn()
        e1.record(s); torch.cuda.synchronize()
        return e0.elapsed_time(e1) / k

    K, W = a.study_steps, max(3, a.warmup)
    for _ in range(W):
        ws.graph_launch()
    l0 = ws.launches()
    if world > 1:
        dist.barrier()
    ms_graph = max_over_ranks(timed(ws.graph_launch, K), world, dev)
    launches_per_step = (ws.launches() - l0) / K
    inf = ws.info()

    def eager():
        ws.leapfrog_step(x, v, m, acc, tau, phi=phi)
        ws.diagnostics(x, v, m, phi, out=diag)
    ms_eager = max_over_ranks(timed(eager, max(3, K // 5)), world, dev)
    steps_run = W + K + max(3, K // 5)
    d1 = ws.diagnostics_segments(x, v, m, phi).cpu().numpy()
    e0_, e1_ = d0[:, 0] + d0[:, 1], d1[:, 0] + d1[:, 1]
    drift = np.abs(e1_ - e0_) / np.abs(e0_)
    if world > 1:
        # per-cluster drifts from every rank
        dt = torch.tensor(drift, dtype=torch.float64, device=dev)
        parts = [torch.zeros(1, dtype=torch.float64, device=dev) for _ in range(world)]
        dist.all_gather(parts, dt.max().reshape(1))
        drift_max = float(torch.stack(parts).max())
    else:
        drift_max = float(drift.max())
    pairs = float(inf["pp_pairs"] + inf["pc_pairs"])
    if world > 1:
        tp = torch.tensor([pairs], dtype=torch.float64, device=dev)
        dist.all_reduce(tp)
        pairs = float(tp.item())
    n, B = n_all, 512
    row = {"study": "ensemble", "clusters": B, "n": n, "n_gpus": world, "scaling": "weak",
           "eps": 0.01, "theta": 0.6, "order": "quadrupole",
           "dtype": "f32+kahan", "tau": tau, "autotuned": {"leaf_cap": best.leaf_cap, "group_size": best.group_size,
                                                           "stack_depth": best.stack_depth},
           "autotune_table": [list(r) for r in table], "autotune_s": tune_s,
           "graph": {"ms_per_step": ms_graph, "particles_per_s": n / (ms_graph / 1e3),
                     "interactions_per_s": pairs / (ms_graph / 1e3),
                     "kernels_per_step": launches_per_step, "steps": K},
           "eager": {"ms_per_step": ms_eager, "particles_per_s": n / (ms_eager / 1e3)},
           "interactions_per_particle": pairs / n, "n_groups (rank 0)": inf["n_groups"],
           "energy_drift_per_cluster": {"median (rank 0)": float(np.median(drift)), "max": drift_max,
                                        "steps": steps_run},
           "status": ws.status()}
    if rank == 0:
        print(json.dumps(row), flush=True)
    if world > 1:
        dist.destroy_process_group()


def study_adjoint(a):
    """Adjoint configuration: Plummer N = 262,144, eps = 0.01, theta = 0.7, quadrupole, K = 16 KDK steps of
    tau = 0.01, checkpoints every 4; loss = sum over the first 1024 particles (caller order) of |x_i^K|^2 + W_K.
    Reports forward and backward times in FP32 and FP64 (and their ratio), the FP32 gradient against the FP64
    one, the theta = 0.7 gradient against the theta = 0 one (every pair exact: the gradient of the direct-sum
    map, FP32), and central differences (h = 1e-6; masses relative 1e-4) of the FP64 GPU map, tree rebuilt
    every step, on 32 coordinates, with the fraction whose perturbation changed the tree structure (node,
    group or pair counts of any step)."""
    import numpy as np
    import torch

    from paper_2412_01733_gb300 import build, inputs, treegb
    from paper_2412_01733_gb300.autograd import TreeLeapfrog
    build.build()
    n, K, tau, nsel, ck = 262144, 16, 0.01, 1024, 4
    x0, v0, m0 = inputs.plummer(n, SEED, device="cuda", dtype=torch.float64)

    def grads(dt, theta):
        ws = treegb.Workspace(n, eps=0.01, theta=theta, order=2, precision="f64" if dt == torch.float64 else "f32")
        x = x0.to(dt).clone().requires_grad_(True)
        v = v0.to(dt).clone().requires_grad_(True)
        m = m0.to(dt).clone().requires_grad_(True)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.synchronize(); e[0].record()
        xK, vK, WK = TreeLeapfrog.apply(x, v, m, ws, K, tau, ck)
        loss = (xK[:, :nsel].double() ** 2).sum() + WK
        e[1].record()
        torch.cuda.synchronize()
        ws.timing(True)
        loss.backward()
        e[2].record(); torch.cuda.synchronize()
        phases, _ = ws.timing_read()
        ws.timing(False)
        st = ws.status()
        out = dict(loss=float(loss), fwd_ms=e[0].elapsed_time(e[1]), bwd_ms=e[1].elapsed_time(e[2]), status=st,
                   bwd_phase_ms={k: round(v[0], 2) for k, v in phases.items() if v[1]})
        g = [t.grad.double() for t in (x, v, m)]
        del ws
        torch.cuda.empty_cache()
        return out, g

    def cmp(g, ref):
        res = {}
        for name, a_, b_ in zip(("x", "v", "m"), g, ref):
            d = (a_ - b_).abs()
            sc = b_.abs().max()
            big = b_.abs() > 1e-3 * sc
            res[name] = {"max_abs_over_max": float(d.max() / sc),
                         "median_rel": float((d[big] / b_.abs()[big]).median())}
        return res

    row = {"study": "adjoint", "n": n, "steps": K, "tau": tau, "eps": 0.01, "theta": 0.7, "checkpoint_every": ck,
           "loss": "sum_{i<1024} |x_i^K|^2 + W_K"}
    r32, g32 = grads(torch.float32, 0.7)
    r64, g64 = grads(torch.float64, 0.7)
    r0, g0 = grads(torch.float32, 0.0)
    row["f32"] = dict(r32, bwd_over_fwd=r32["bwd_ms"] / r32["fwd_ms"])
    row["f64"] = dict(r64, bwd_over_fwd=r64["bwd_ms"] / r64["fwd_ms"])
    row["theta0_f32"] = dict(r0, bwd_over_fwd=r0["bwd_ms"] / r0["fwd_ms"])
    row["f32_vs_f64"] = cmp(g32, g64)
    row["tree_vs_theta0"] = cmp(g32, g0)

    ws = treegb.Workspace(n, eps=0.01, theta=0.7, order=2, precision="f64")

    def L(xx, vv, mm):
        xx, vv = xx.clone(), vv.clone()
        acc, phi = ws.accel(xx, mm)
        sig = []
        for _ in range(K):
            ws.leapfrog_step(xx, vv, mm, acc, tau, phi=phi)
            inf = ws.info()
            sig.append((inf["n_nodes"], inf["n_groups"], inf["pp_pairs"], inf["pc_pairs"]))
        return float((xx[:, :nsel] ** 2).sum() + ws.diagnostics(xx, vv, mm, phi)[1]), sig

    L0, sig0 = L(x0, v0, m0)
    rng = np.random.default_rng(3)
    ok = changed = 0
    rows = []
    for k in range(32):
        which, d, i = k % 3, int(rng.integers(0, 3)), int(rng.integers(0, n))
        if which == 2:
            h = 1e-4 * float(m0[i])
            mp = m0.clone(); mp[i] += h; mn = m0.clone(); mn[i] -= h
            (Lp, sp), (Ln, sn) = L(x0, v0, mp), L(x0, v0, mn)
            g = float(g64[2][i])
        else:
            h = 1e-6
            base = x0 if which == 0 else v0
            bp = base.clone(); bp[d, i] += h; bn = base.clone(); bn[d, i] -= h
            (Lp, sp), (Ln, sn) = (L(bp, v0, m0), L(bn, v0, m0)) if which == 0 else (L(x0, bp, m0), L(x0, bn, m0))
            g = float(g64[which][d, i])
        fd = (Lp - Ln) / (2 * h)
        noise = 20 * 2.2e-16 * abs(L0) / (2 * h)
        good = abs(fd - g) <= 1e-5 * abs(g) + noise
        ch = sp != sig0 or sn != sig0
        ok += good; changed += ch
        rows.append({"coord": ["x", "v", "m"][which], "d": d, "i": i, "fd": fd, "grad": g, "match": bool(good),
                     "structure_changed": bool(ch)})
    row["fd_unfrozen_f64"] = {"coordinates": 32, "match_1e-5": ok, "structure_changed": changed,
                              "loss": L0, "detail": rows}
    print(json.dumps(row), flush=True)


def study_plain(a):
    """Plain FP64 configuration: Plummer N = 16384 (G = M = a = 1), eps = 0.01, theta = 0.7, monopole cells,
    leaf <= 16; one force evaluation and 10 KDK steps of tau = 0.01 on the GPU (FP64 walk) and with the
    oracle.  Reports the tree force error against the FP64 direct sum (all particles), the GPU against the
    oracle, and the energy and momentum drift of both runs."""
    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2412_01733_gb300 import build, inputs, treegb
    build.build()
    n, eps, theta, tau, K = 16384, 0.01, 0.7, 0.01, 10
    x, v, m = inputs.plummer(n, SEED)
    xn, vn, mn = x.numpy(), v.numpy(), m.numpy()
    kw = dict(eps=eps, theta=theta, lcap=16, gs=32, quad=False)
    ad, pd = O.direct(xn, mn, eps=eps)
    ref = O.tree_forces(xn, mn, **kw)
    ws = treegb.Workspace(n, precision="f64", eps=eps, theta=theta, order=0, leaf_cap=16, group_size=32)
    xg, vg, mg = x.cuda().contiguous(), v.cuda().contiguous(), m.cuda().contiguous()
    ag, pg = ws.accel(xg, mg)
    agn = ag.cpu().numpy()
    e_tree = np.linalg.norm(ref.a - ad, axis=0) / np.linalg.norm(ad, axis=0)
    e_gpu = np.linalg.norm(agn - ref.a, axis=0) / np.linalg.norm(ref.a, axis=0)
    d0 = O.diagnostics(xn, vn, mn, ref.phi)
    acc = lambda xx: O.tree_accel(xx, mn, **kw)
    xo, vo, ao, po = O.kdk(xn, vn, mn, tau, K, acc, a0=(ref.a, ref.phi))
    d1 = O.diagnostics(xo, vo, mn, po)
    g0 = ws.diagnostics(xg, vg, mg, pg).cpu().numpy()
    for _ in range(K):
        ws.leapfrog_step(xg, vg, mg, ag, tau, phi=pg)
    g1 = ws.diagnostics(xg, vg, mg, pg).cpu().numpy()
    pscale = float(np.sum(mn * np.linalg.norm(vn, axis=0)))
    row = {"study": "plain", "n": n, "eps": eps, "theta": theta, "order": "monopole", "precision": "f64",
           "tree_vs_direct": {"median": float(np.median(e_tree)), "p99": float(np.quantile(e_tree, 0.99)),
                              "max": float(e_tree.max())},
           "gpu_vs_oracle": {"median": float(np.median(e_gpu)), "max": float(e_gpu.max())},
           "oracle_kdk": {"energy_drift": abs(d1["etot"] - d0["etot"]) / abs(d0["etot"]),
                          "momentum_drift": float(np.abs(d1["P"] - d0["P"]).max()) / pscale},
           "gpu_kdk": {"energy_drift": float(abs((g1[0] + g1[1]) - (g0[0] + g0[1])) / abs(g0[0] + g0[1])),
                       "momentum_drift": float(np.abs(g1[2:5] - g0[2:5]).max()) / pscale},
           "gpu_vs_oracle_after_kdk": float(np.abs(xg.cpu().numpy() - xo).max()),
           "status": ws.status()}
    print(json.dumps(row), flush=True)


def main():
    a = _args()
    if a.study == "plain":
        return study_plain(a)
    if a.study == "theta":
        return study_theta(a)
    if a.study == "adjoint":
        return study_adjoint(a)
    if a.study == "ensemble":
        return study_ensemble(a)
    if a.study == "threads":
        return study_threads(a)
    if a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)


if __name__ == "__main__":
    main()
