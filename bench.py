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
# Algorithmic flop counts per pair: PP with potential 20; quadrupole PC 60, the
# low end of the 60-65 flop estimate of the method's per-interaction work (Qy
# 9 operations, yQy 3, five scalar coefficients, 3 x 2 accumulating FMAs);
# monopole PC 20.  The pair terms as written (FMA = 2 flops, rsqrt = 1) do 54
# flops per quadrupole PC pair; the fraction at that count is reported too.
FLOPS_PP, FLOPS_PC_QUAD, FLOPS_PC_MONO = 20, 60, 20
FLOPS_PC_QUAD_AS_WRITTEN = 54
# FP32 peak derived from unit counts and clocks: 152 SMs x 128 FP32 lanes x
# 2 flops (FMA) x 2.070 GHz.
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.070e9 / 1e12
# DRAM bytes per walk launch from ncu (dram__bytes_read.sum + write.sum) on the
# N = 1e7 galaxy case of the same kernel, per particle (scaled by N below);
# None when the kernel has changed since the counters were taken.
WALK_DRAM_BYTES_PER_PARTICLE = 716
WALK_TRAFFIC_SOURCE = "ncu dram__bytes_read.sum + dram__bytes_write.sum of k_walk, galaxy N=1e7, scaled by N"



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
    ap.add_argument("--err-samples-fp64", type=int, default=1024,
                    help="of those, particles whose direct sum is also taken in FP64 (reference check)")
    ap.add_argument("--parity-groups", type=int, default=3000,
                    help="walk groups whose lists and forces the FP64 oracle evaluates in the CPU-baseline leg "
                         "(the oracle's box, keys, order, octree, moments and groups always cover all N)")
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
    x, v, m, comp = inputs.galaxy(n, SEED + rank, device=dev, dtype=torch.float32, return_component=True)
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
    flops_written = FLOPS_PP * inf["pp_pairs"] + FLOPS_PC_QUAD_AS_WRITTEN * inf["pc_pairs"]
    achieved = flops / walk_s / 1e12
    traffic = None if WALK_DRAM_BYTES_PER_PARTICLE is None else WALK_DRAM_BYTES_PER_PARTICLE * n
    fp32_scalar, fp32_packed = treegb.fp32_peak()
    roofline = {"bound": "alu", "kernel": "k_walk<float,1,quad,kahan,soft,force>", "achieved": achieved,
                "peak": FP32_PEAK_TFLOPS, "unit": "TFLOP/s", "frac": achieved / FP32_PEAK_TFLOPS,
                "traffic": traffic, "traffic_source": WALK_TRAFFIC_SOURCE if traffic is not None else
                "not captured for the current kernel",
                "peak_source": "derived: 152 SM x 128 FP32 lanes x 2 flops x 2.07 GHz (MEASURED_PEAKS has no FP32 "
                               "entry)",
                "flops_per_pair": {"pp": FLOPS_PP, "pc_quadrupole": FLOPS_PC_QUAD},
                "measured_fp32_peak": {"scalar_ffma": fp32_scalar, "packed_ffma2": fp32_packed,
                                       "frac_vs_packed": achieved / fp32_packed},
                "frac_at_as_written_flops": flops_written / walk_s / 1e12 / FP32_PEAK_TFLOPS,
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
        # end to end through the C ABI with host-resident state (first among the extras, right after
        # the timed steps): leapfrog_step_host copies the state x, v, m, a up, runs the step and the
        # diagnostics; the new x comes back by a copy under the tree build and walk, v and a by the
        # walk's own stores into the (mapped, pinned) host arrays, the diagnostics (which carry W) by a
        # copy after the step
        xh = x.cpu().pin_memory(); vh = v.cpu().pin_memory(); mh = m.cpu().pin_memory()
        ah = acc.cpu().pin_memory()
        dh = torch.empty(8, dtype=torch.float64).pin_memory()
        ws.leapfrog_step_host(xh, vh, mh, ah, TAU, diag=dh)
        torch.cuda.synchronize()
        barrier()
        clocks_e2e = Clocks(local)
        clocks_e2e.start()
        ws.timing(True)
        h0 = torch.cuda.Event(enable_timing=True); h1 = torch.cuda.Event(enable_timing=True)
        h0.record(stream)
        for _ in range(a.steps):
            ws.leapfrog_step_host(xh, vh, mh, ah, TAU, diag=dh)
        h1.record(stream)
        torch.cuda.synchronize()
        barrier()
        ck_e2e = clocks_e2e.stop()
        te = max_over_ranks(h0.elapsed_time(h1) / 1e3, world, dev)
        ph_e2e, _ = ws.timing_read()
        ws.timing(False)
        if ws.status() != 0:
            raise RuntimeError("device status set in the end-to-end steps")
        split = {"h2d_ms": ph_e2e["h2d"][0] / a.steps, "d2h_after_walk_ms": ph_e2e["d2h"][0] / a.steps,
                 "walk_ms": ph_e2e["walk"][0] / a.steps, "step_ms": te * 1e3 / a.steps}
        out["e2e"] = {"value": world * n * a.steps / te, "unit": UNIT,
                      "h2d_bytes_per_step": 40 * n, "d2h_bytes_per_step": 36 * n + 64, "clocks": ck_e2e,
                      "api": "leapfrog_step_host (pinned host arrays; x copied back on a second stream under "
                             "the tree build and walk; v and a written into the mapped host arrays by the walk "
                             "itself, so d2h_after_walk_ms is the diagnostics' copy)",
                      "per_step": {k: round(v, 2) for k, v in split.items()}}
        # continue from the host state: the device arrays take it back
        x.copy_(xh); v.copy_(vh); acc.copy_(ah)
        torch.cuda.synchronize()
        del xh, vh, mh, ah, dh
        # force error of the FP32 tree against the GPU FP64 direct sum of Eq. 1 (sampled particles;
        # the state after the end-to-end steps, whose accelerations belong to these positions)
        out["force_err_vs_direct"] = force_error(ws, x, m, acc, comp, a.err_samples, a.err_samples_fp64)
        tgt = out["force_err_vs_direct"].pop("_targets")
        # same-GPU FP64 plain path: one force evaluation (build + moments + walk) on the same state
        x64, m64 = x.double().contiguous(), m.double().contiguous()
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
        # the FP64 CPU oracle on the host cores, rank 0 at N = 1 only: the full canonical tree of this
        # state over all N particles, lists and forces for sampled groups (rate extrapolated), compared
        # with the GPU's tree, lists and forces
        if world == 1:
            out["cpu_baseline"], out["oracle_parity_1e8"] = cpu_baseline_full(ws, x, m, a.parity_groups)
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


def force_error(ws, x, m, acc, comp, nsamp, nsamp64):
    """Relative error |a_tree - a_direct| / |a_direct| of the FP32 tree accelerations on nsamp seeded
    particles against the GPU direct sum of Eq. 1 (FP32 pair terms, compensated sums, FP64 chunk totals),
    the first nsamp64 of them also against the FP64 direct sum (which bounds the reference's own error),
    with the tail broken down by galaxy component and by |a|, and, for the 100 worst particles, the
    cancellation ratio sum_j |a_ij| / |a_i| (a_ij the pair terms of Eq. 1, summed in FP64)."""
    import torch
    n = x.shape[1]
    dev = x.device
    g = torch.Generator().manual_seed(SEED)
    tgt = torch.randint(0, n, (min(n, nsamp),), generator=g).to(dev)
    e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
    e2 = torch.cuda.Event(enable_timing=True)
    e0.record()
    ad, _ = ws.direct(x, m, tgt, precision="f32")
    e1.record()
    x64, m64 = x.double().contiguous(), m.double().contiguous()
    t64 = tgt[:nsamp64]
    a64, _ = ws.direct(x64, m64, t64, precision="f64")
    e2.record()
    torch.cuda.synchronize()
    at = acc[:, tgt].double()
    an = ad.norm(dim=0)
    err = ((at - ad).norm(dim=0) / an)
    q = lambda v: {"median": float(v.median()), "p99": float(v.quantile(0.99)), "max": float(v.max()),
                   "count": int(v.numel())}
    ref_dev = ((ad[:, :nsamp64] - a64).norm(dim=0) / a64.norm(dim=0))
    err64 = ((at[:, :nsamp64] - a64).norm(dim=0) / a64.norm(dim=0))
    out = {"samples": int(tgt.numel()),
           "reference": "GPU direct sum of Eq. 1: FP32 pair terms, compensated sums, FP64 chunk totals",
           "direct_ms": e0.elapsed_time(e1), **q(err),
           "fp64_check": {"samples": int(t64.numel()), "direct_fp64_ms": e1.elapsed_time(e2),
                          "reference_max_rel_dev_from_fp64": float(ref_dev.max()),
                          "error_vs_fp64": q(err64)}}
    names = ("disc", "bulge", "halo")
    c = comp[tgt]
    out["by_component"] = {names[k]: q(err[c == k]) for k in range(3) if int((c == k).sum()) > 0}
    qs = torch.quantile(an, torch.tensor([0.2, 0.4, 0.6, 0.8], dtype=torch.float64, device=dev))
    edges = [0.0] + [float(v) for v in qs] + [float("inf")]
    out["by_accel_quintile"] = [dict(q(err[(an >= lo) & (an < hi)]), a_lo=lo, a_hi=hi)
                                for lo, hi in zip(edges[:-1], edges[1:])]
    worst = torch.argsort(err, descending=True)[:100]
    eps2 = PARAMS["eps"] ** 2
    ratios = []
    for w in worst.tolist():
        i = int(tgt[w])
        d = x64 - x64[:, i:i + 1]
        r2 = (d * d).sum(dim=0) + eps2
        t = m64 * d.norm(dim=0) / (r2 * r2.sqrt())
        t[i] = 0.0
        ratios.append(float(t.sum()) / float(an[w]))
    rw = torch.tensor(ratios, dtype=torch.float64)
    r_all = x64[:, tgt[worst]].norm(dim=0)
    out["worst100"] = {"err_min": float(err[worst].min()), "sum_abs_terms_over_a": {
        "median": float(rw.median()), "min": float(rw.min()), "max": float(rw.max())},
        "component_counts": {names[k]: int((c[worst] == k).sum()) for k in range(3)},
        "radius_median": float(r_all.median())}
    out["_targets"] = tgt
    return out


def _segment_sorted(off, vals):
    """Entries of each CSR segment in ascending order (segments kept in place)."""
    import numpy as np
    off = np.asarray(off, np.int64)
    g = np.repeat(np.arange(len(off) - 1, dtype=np.int64), np.diff(off))
    return np.sort((g << 32) | np.asarray(vals, np.int64)) & 0xffffffff


def cpu_baseline_full(ws, x, m, ngroups_sample):
    """The FP64 CPU oracle on the host cores, on the benchmark's own state: the canonical tree (box,
    keys, order, octree, moments, walk groups) over all N particles, then lists and forces for
    ngroups_sample seeded walk groups.  Returns (cpu_baseline, parity):
      cpu_baseline  particles/s of one oracle force evaluation, extrapolated from the sample as
                    N / (T_tree + T_walk(sample) * N / sample particles);
      parity        the GPU's sorted keys, permutation, node arrays and groups against the oracle's
                    (bit-exact), FP64 moments (rounding), the sampled groups' interaction lists (as
                    sets, exact) and FP32 forces against the oracle's on the same tree."""
    import numpy as np
    import torch

    from oracle import oracle as O
    n = x.shape[1]
    inf = ws.info()
    ng = inf["n_groups"]
    rng = np.random.default_rng(SEED)
    sel = np.sort(rng.choice(ng, size=min(ng, ngroups_sample), replace=False)).astype(np.int64)
    # GPU: the stored tree of this state, its lists (stored by this walk) and FP32 forces
    a_g, phi_g = ws.forces(emit_lists=True)
    torch.cuda.synchronize()
    ex = ws.export_tree()
    gf_g = ws.export_groups().cpu().numpy()
    M_g, R_g, Q_g = (t.cpu().numpy() for t in ws.export_moments())
    pco, pcl, ppo, ppl = ws.export_lists_groups(sel)
    pcl, ppl = pcl.cpu().numpy(), ppl.cpu().numpy()
    keys_g = ex["keys"].cpu().numpy().view(np.uint64)
    perm_g = ex["perm"].cpu().numpy().view(np.uint32).astype(np.int64)
    nodes_g = {k: ex[k].cpu().numpy() for k in ("level", "corner", "first", "count", "child", "nchild")}
    xh = x.double().cpu().numpy(); mh = m.double().cpu().numpy()
    # oracle
    T = {}
    t0 = time.perf_counter()
    ref = O.tree_forces(xh, mh, eps=PARAMS["eps"], theta=PARAMS["theta"], lcap=PARAMS["leaf_cap"],
                        gs=PARAMS["group_size"], quad=True, groups_sel=sel, timings=T)
    t_oracle = time.perf_counter() - t0
    t_tree = sum(T[k] for k in ("box", "keys", "sort", "octree", "moments", "groups"))
    t_walk = T["lists"] + T["forces"]
    gf = ref.gfirst
    idx = np.concatenate([ref.perm[gf[g]: gf[g + 1]] for g in sel])
    cpu = {"value": n / (t_tree + t_walk * n / len(idx)), "unit": UNIT, "cores": O.threads(), "kind": "oracle",
           "sample": (f"FP64 oracle on this run's state at N={n}: canonical tree over all particles "
                      f"({t_tree:.1f} s), lists + forces for {len(sel)} seeded walk groups = {len(idx)} particles "
                      f"({t_walk:.1f} s); rate extrapolated to all N (tree stages are single-threaded except "
                      f"keys, moments and groups)"),
           "stages_s": {k: round(v, 2) for k, v in T.items()}}
    # structure, bit for bit
    t = ref.tree
    same = lambda a, b: bool(a.shape == b.shape and np.array_equal(a, b))
    nn_ok = int(inf["n_nodes"]) == t.nn
    checks = {
        "keys": same(keys_g, ref.key[ref.perm]),
        "perm": same(perm_g, ref.perm),
        "n_nodes": nn_ok,
        "level": nn_ok and same(nodes_g["level"].astype(np.int64), t.level.astype(np.int64)),
        "corner": nn_ok and same(nodes_g["corner"].view(np.uint32), t.corner),
        "first": nn_ok and same(nodes_g["first"].astype(np.int64), t.first),
        "count": nn_ok and same(nodes_g["count"].astype(np.int64), t.count),
        "child": nn_ok and same(nodes_g["child"].astype(np.int64), t.child),
        "nchild": nn_ok and same(nodes_g["nchild"].astype(np.int64), t.nchild.astype(np.int64)),
        "groups": same(gf_g.astype(np.int64), gf),
    }
    side = np.ldexp(1.0, ref.k - t.level.astype(np.int64))
    mom = {}
    if nn_ok:
        mom = {"M_rel": float(np.max(np.abs(M_g - ref.M) / np.maximum(np.abs(ref.M), 1e-300))),
               "R_over_L": float(np.max(np.abs(R_g - ref.R)) / np.ldexp(1.0, ref.k)),
               "Q_over_Ms2": float(np.max(np.abs(Q_g - ref.Q) / (np.abs(ref.M) * side * side + 1e-300)))}
    lists_ok = (same(np.asarray(pco, np.int64), ref.pc_off) and same(np.asarray(ppo, np.int64), ref.pp_off)
                and same(_segment_sorted(pco, pcl), ref.pc_list) and same(_segment_sorted(ppo, ppl), ref.pp_list))
    # forces of the sampled groups' particles: GPU FP32 against the oracle's FP64 on the same tree
    ia = torch.as_tensor(idx, device=x.device)
    ag = a_g[:, ia].double().cpu().numpy(); pg = phi_g[ia].double().cpu().numpy()
    ar = ref.a[:, idx]; pr = ref.phi[idx]
    e = np.linalg.norm(ag - ar, axis=0) / np.linalg.norm(ar, axis=0)
    ep = np.abs(pg - pr) / np.abs(pr)
    parity = {"groups": int(len(sel)), "particles": int(len(idx)), "n": n,
              "structure_exact": bool(all(checks.values())), "structure": checks,
              "moments_fp64": mom, "moments_ok": bool(mom and mom["M_rel"] <= 1e-12 and mom["R_over_L"] <= 1e-12
                                                        and mom["Q_over_Ms2"] <= 1e-10),
              "lists_exact": bool(lists_ok), "pc_entries": int(pco[-1]), "pp_leaves": int(ppo[-1]),
              "median": float(np.median(e)), "max": float(e.max()),
              "phi_median": float(np.median(ep)), "phi_max": float(ep.max()),
              "tolerance": "median <= 1e-5, max <= 1e-4 (FP32 against FP64 on the same tree)",
              "within_tolerance": bool(np.median(e) <= 1e-5 and e.max() <= 1e-4),
              "oracle_s": round(t_oracle, 1)}
    # the GPU FP64 direct sum of Eq. 1 (the error reference of the force-error check) against the
    # oracle's own direct sum, on 256 of the sampled particles (about 12 s of oracle time at N = 1e8)
    t64 = np.ascontiguousarray(idx[:: max(1, len(idx) // 256)][:256])
    x64, m64 = x.double().contiguous(), m.double().contiguous()
    ad_g, pd_g = ws.direct(x64, m64, torch.as_tensor(t64, device=x.device), precision="f64")
    t0 = time.perf_counter()
    ad_o, pd_o = O.direct(xh, mh, G=1.0, eps=PARAMS["eps"], targets=t64)
    t_dir = time.perf_counter() - t0
    ad_g = ad_g.cpu().numpy(); pd_g = pd_g.cpu().numpy()
    parity["direct_fp64_vs_oracle"] = {
        "targets": int(len(t64)), "oracle_s": round(t_dir, 1),
        "max_rel": float(np.max(np.linalg.norm(ad_g - ad_o, axis=0) / np.linalg.norm(ad_o, axis=0))),
        "phi_max_rel": float(np.max(np.abs(pd_g - pd_o) / np.abs(pd_o)))}
    if e.max() > 1e-4:
        # offending particles: how strongly the terms of their direct sum cancel
        eps2 = PARAMS["eps"] ** 2
        bad = []
        for j in np.argsort(-e)[:10]:
            i = int(idx[j])
            d = x64 - x64[:, i:i + 1]
            r2 = (d * d).sum(dim=0) + eps2
            tt = m64 * d.norm(dim=0) / (r2 * r2.sqrt())
            tt[i] = 0.0
            bad.append({"err": float(e[j]), "sum_abs_terms_over_a": float(tt.sum()) / float(np.linalg.norm(ar[:, j]))})
        parity["worst"] = bad
    del pcl, ppl, ref
    return cpu, parity


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
    force evaluation (mean and standard error over 10 evaluations after one warm-up, the paper's Sec. 3
    timing method), and the relative energy drift over K KDK steps (tau = 0.005; K = 100 by default, for
    both precisions)."""
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

    def timed(fn, reps=10):
        """One warm-up call, then reps timed calls: (last output, mean ms, standard error of the mean)."""
        fn()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(reps + 1)]
        ev[0].record()
        for k in range(reps):
            out = fn()
            ev[k + 1].record()
        torch.cuda.synchronize()
        t = [ev[k].elapsed_time(ev[k + 1]) for k in range(reps)]
        mean = sum(t) / reps
        sem = statistics.stdev(t) / math.sqrt(reps) if reps > 1 else 0.0
        return out, mean, sem

    for theta in (0.4, 0.5, 0.7, 1.0):
        row = {"study": "theta", "n": n, "eps": eps, "theta": theta, "order": "quadrupole", "leaf_cap": 16}
        for prec, dt in (("f32", torch.float32), ("f64", torch.float64)):
            # explicit copies: the leapfrog below advances them in place
            xs, vs, ms = x.to(dt).clone(), v.to(dt).clone(), m.to(dt).clone()
            ws = treegb.Workspace(n, precision=prec, eps=eps, theta=theta)
            (acc, phi), ms_force, ms_sem = timed(lambda: ws.accel(xs, ms))
            e = ((acc[:, tgt].double() - a_ref).norm(dim=0) / a_ref.norm(dim=0)).cpu()
            inf = ws.info()
            row[prec] = {"force_ms": ms_force, "force_ms_sem": ms_sem, "force_reps": 10,
                         "particles_per_s": n / (ms_force / 1e3),
                         "err_median": float(e.median()), "err_p99": float(e.quantile(0.99)),
                         "err_max": float(e.max()), "interactions_per_particle": (inf["pp_pairs"] + inf["pc_pairs"]) / n}
            steps = a.study_steps
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
    E = S/M, for M host threads, galaxy recipe at N = 1e5, 1e6 and 1e7, theta = 1, and E against N at M = 4
    for N = 2^17 .. 2^24."""
    import os as _os

    import numpy as np
    import torch

    from oracle import oracle as O
    from paper_2412_01733_gb300 import inputs
    ncpu = _os.cpu_count() or 1
    ms_list = sorted({1, 2, 4, 8, ncpu // 2, ncpu} - {0})
    for n in (100_000, 1_000_000, 10_000_000):
        x, _, m = inputs.galaxy(n, SEED, dtype=torch.float64)
        x, m = x.numpy(), m.numpy()
        res = {}
        # N = 1e7: one evaluation per thread count (about 200 s on one Grace core), at 1, 4 and all threads
        for M in (ms_list if n <= 1_000_000 else sorted({1, 4, ncpu})):
            O.set_threads(M)
            reps = 10 if n <= 100_000 else (5 if n <= 1_000_000 else 1)
            ts = []
            for _ in range(reps):
                t0 = time.perf_counter()
                O.tree_forces(x, m, eps=PARAMS["eps"], theta=1.0, lcap=PARAMS["leaf_cap"], gs=PARAMS["group_size"])
                ts.append(time.perf_counter() - t0)
            ts = np.array(ts)
            res[M] = (ts.mean(), ts.std(ddof=1) / np.sqrt(len(ts)) if len(ts) > 1 else 0.0)
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
    # efficiency against N at M = 4 threads (the paper's E(N) view), N = 2^17 .. 2^24 (one evaluation
    # per thread count above 2^21)
    for lg in range(17, 25):
        n = 1 << lg
        x, _, m = inputs.galaxy(n, SEED, dtype=torch.float64)
        x, m = x.numpy(), m.numpy()
        T = {}
        for M in (1, 4):
            O.set_threads(M)
            ts = []
            for _ in range(2 if lg <= 21 else 1):
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
    best, table = treegb.autotune(x, m, offsets=off, reps=3, max_err=1e-3, **base)
    tune_s = time.perf_counter() - t0
    chosen_err = next(r[4] for r in table
                      if (int(r[0]), int(r[1]), int(r[2])) == (best.leaf_cap, best.group_size, best.stack_depth))
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
                                                           "stack_depth": best.stack_depth,
                                                           "median_force_err": chosen_err, "max_err": 1e-3},
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
