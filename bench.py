"""Benchmark of the periodic QEq solve on one B300 (or N replicas).

One step = one complete cold-start QEq solve of the workload cell through the
C ABI (charges to 1e-5 e, final FP64 residual check included), inputs resident
on the device.  The default workload is the 13,824-atom rock-salt cell
(12x12x12 conventional cells, jitter 0.15 A, r_cut 8 A, ewald_tol 1e-6); the
chosen form is mixed precision (FP32 mesh, FP64 reductions) with the PCG
iterations captured in a CUDA graph.  Beside it: the plain FP64 GPU PCG (no
graph), the roofline of the dominant matvec kernel (CUDA events on the plan's
stream), an end-to-end number through the public API with host buffers, and
the FP64 CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 2|1|3|5]

--gpus N > 1 runs under torch.distributed.run with no collective on the data
path: a single cell runs as one replica per rank ("scaling": "weak"); the
512-structure batch is split across ranks by the greedy largest-first rule of
paper_2607_17978_b300/shard.py ("scaling": "strong").  value = all ranks'
solves / max-over-ranks time.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "QEq solves/s and atoms*CG-iters/s at 1e-5 e vs plain FP64 GPU PCG; % HBM roofline"
UNIT = "solves/s"
# Jacobi-PCG iterations of a full solve of the default workload at 1e-5 e (about 100 on
# this 13,824-atom cell), used to
# extrapolate the CPU oracle's matvec time to a solve (the oracle's own solve is
# a dense LU that does not fit the time budget at this size).
PCG_ITERS_REFERENCE = 100
WORKLOAD_OPTS = {
    1: dict(ewald_tol=1e-7, r_cut=9.0),
    2: dict(ewald_tol=1e-6, r_cut=8.0),
    3: dict(ewald_tol=1e-6, r_cut=8.0),
    4: dict(ewald_tol=1e-6, r_cut=8.0),
    5: dict(ewald_tol=1e-6, r_cut=8.0),
}
WORKLOAD_NAME = {
    1: "rocksalt 3x3x3 (216 atoms), chi_A~N(-2,.3) chi_B~N(2,.3), J 2/1.5, sigma 1.0/1.8, r_cut 9, ewald_tol 1e-7",
    2: "rocksalt 12x12x12 (13,824 atoms), jitter 0.15 A, r_cut 8 A, ewald_tol 1e-6",
    3: "rocksalt 24x24x24 -5% vacancies, triclinic shear <=10 deg (105,062 atoms), r_cut 8, ewald_tol 1e-6",
    4: ("512 uneven periodic cells, N log-uniform 64-4096 (519,537 atoms), density 0.045/A^3, orthorhombic or "
        "triclinic, 2-4 species, chi~N(0,1.5), J~U(1,3), sigma~U(0.8,2.0), q_tot in {-1,0,1}; one batched solve"),
    5: "rocksalt 50x50x50 -2% vacancies, jitter 0.2 A (980,000 atoms), r_cut 8, ewald_tol 1e-6",
}


def workload_structs(w: int):
    from paper_2607_17978_b300 import synth
    return synth.batch_workload(512) if w == 4 else [synth.workload(w)]


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self, index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------- byte model
def stage_bytes(plan, prec: str, n_atoms: int, pairs: int):
    """Algorithmic DRAM bytes per launch of each matvec stage (all structures of the plan)."""
    cs = 8 if prec == "mixed" else 16          # complex element
    rs = 4 if prec == "mixed" else 8           # real element
    mesh = 0
    for s in range(plan.n_struct):
        qi = plan.query(s)
        K = qi["mesh"]
        mesh += K[0] * K[1] * K[2] * ((qi["n_species"] + 1) // 2)
    p = plan.query(0)["spline_order"]
    atom_in = n_atoms * (3 * p * rs + 4 + 4 + 8)  # spline weights, stencil base, species, x
    return {
        "species_sums": n_atoms * (8 + 4),
        "spread": mesh * cs + atom_in,
        "fft_z": 2 * mesh * cs,
        "fft_y": 2 * mesh * cs,
        "fft_x_green": 2 * mesh * cs,
        "ifft_y": 2 * mesh * cs,
        "ifft_z": 2 * mesh * cs,
        "gather": mesh * cs + atom_in + n_atoms * (8 + 8 + 8) + pairs * (rs + 4),
    }


def load_traffic():
    """DRAM traffic per launch of the dominant kernel from the committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- CPU oracle
def cpu_oracle_matvec_time(st, budget_s: float = 20.0):
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    cores = len(os.sched_getaffinity(0))
    os.environ.setdefault("OMP_NUM_THREADS", str(cores))
    O.build_c()
    q = np.random.default_rng(0).normal(size=st.n)
    times = []
    t_start = time.perf_counter()
    while True:
        t0 = time.perf_counter()
        O.ewald_matvec(st.cell, st.pos, st.sigma, q, k_e=synth.COULOMB_K_EV_A)
        times.append(time.perf_counter() - t0)
        if time.perf_counter() - t_start > budget_s * 0.5 or len(times) >= 5:
            break
    return min(times), cores, len(times)


def cpu_oracle_dense_batch(structs, every: int = 64):
    """Dense bordered oracle solves of a stratified sample of a batch: solves/s."""
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    cores = len(os.sched_getaffinity(0))
    O.build_c()
    sample = list(range(0, len(structs), every))
    t0 = time.perf_counter()
    for k in sample:
        O.solve_structure(structs[k], k_e=synth.COULOMB_K_EV_A)
    t = time.perf_counter() - t0
    return (len(sample) / t, cores,
            f"dense FP64 oracle solves (Ewald assembly + bordered LU) of {len(sample)} of {len(structs)} structures "
            f"(every {every}th), {t:.1f} s")


def run_reference(args):
    """The CPU oracle as it stands, timed on the host cores on this workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    structs = workload_structs(args.workload)
    cores = len(os.sched_getaffinity(0))
    O.build_c()
    if len(structs) > 1:
        # one dense bordered solve per step, cycling through every 64th structure
        sample = list(range(0, len(structs), 64))
        for k in range(args.warmup):
            O.solve_structure(structs[sample[k % len(sample)]], k_e=synth.COULOMB_K_EV_A)
        t0 = time.perf_counter()
        for k in range(args.steps):
            O.solve_structure(structs[sample[k % len(sample)]], k_e=synth.COULOMB_K_EV_A)
        solve_s = (time.perf_counter() - t0) / args.steps
        desc = (f"dense FP64 oracle solve (Ewald assembly + bordered LU) of one structure per step, cycling through "
                f"every 64th of the {len(structs)} structures")
        atoms = sum(x.n for x in structs)
    else:
        st = structs[0]
        q = np.random.default_rng(0).normal(size=st.n)
        for _ in range(args.warmup):
            O.ewald_matvec(st.cell, st.pos, st.sigma, q, k_e=synth.COULOMB_K_EV_A)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            O.ewald_matvec(st.cell, st.pos, st.sigma, q, k_e=synth.COULOMB_K_EV_A)
        solve_s = (time.perf_counter() - t0) / args.steps * PCG_ITERS_REFERENCE
        desc = (f"one FP64 Ewald matvec of the full {st.n}-atom cell per step by the CPU oracle, "
                f"x {PCG_ITERS_REFERENCE} PCG iterations (extrapolated to a solve)")
        atoms = st.n
    value = 1.0 / solve_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME[args.workload], "atoms": atoms, "structures": len(structs)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- our arm
def run_profile(args):
    """A few solves of a rock-salt cell of --cells^3 conventional cells (config-5 recipe),
    for ncu captures: no plain-FP64 leg, no end-to-end leg, no CPU oracle."""
    import torch
    from paper_2607_17978_b300 import build, qeq, synth
    build.build()
    st = synth.rocksalt(args.cells, synth.ROCKSALT_A, 0.2, synth.rng_for(5, 1), vacancy_frac=0.02)
    plan = qeq.plan_for_structures([st], precision=args.precision, ewald_tol=1e-6, r_cut=8.0)
    pos, spc, chi, J, qt = qeq.pack([st])
    d = [torch.tensor(a, device="cuda") for a in (pos, spc, chi, J)]
    for _ in range(args.steps):
        r = plan.solve(*d, qt)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": f"rocksalt {args.cells}^3", "atoms": st.n, "mesh": plan.query(0)["mesh"],
                      "iterations": r.info[0]["iterations"], "stages_ms": plan.profile_matvec(5)}))
    return 0


def run_ours(args):
    import torch
    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    from paper_2607_17978_b300 import build, qeq, shard, synth
    build.build()
    structs_all = workload_structs(args.workload)
    # batches of independent structures are split across ranks (greedy largest-first,
    # no data-path collective; total work fixed); a single cell runs as one replica per rank
    sharded = world > 1 and len(structs_all) > 1
    if sharded:
        mine = shard.rank_share([shard.structure_cost(x) for x in structs_all], rank, world)
        structs = [structs_all[i] for i in mine]
    else:
        structs = structs_all
    n_struct = len(structs)
    n_atoms = sum(x.n for x in structs)
    n_total = len(structs_all) if sharded else world * n_struct
    atoms_total = sum(x.n for x in structs_all) if sharded else n_atoms
    st = structs[0]
    opts = WORKLOAD_OPTS[args.workload]
    pos, spc, chi, J, qt = qeq.pack(structs)
    d_pos = torch.tensor(pos, device=dev)
    d_spc = torch.tensor(spc, device=dev)
    d_chi = torch.tensor(chi, device=dev)
    d_J = torch.tensor(J, device=dev)
    plan = qeq.plan_for_structures(structs, precision=args.precision, device=dev, preconditioner=args.precond, **opts)
    q_out = torch.empty(n_atoms, dtype=torch.float64, device=dev)
    # learned warm start for the rock-salt workloads of the recipe the network was trained on
    # (unsheared, jittered, few vacancies; the sheared 5%-vacancy cell of workload 3 is outside it)
    warm = args.warm
    model = os.path.join(ROOT, "paper_2607_17978_b300", "models", "warmstart_rocksalt.npz")
    if warm == "auto":
        warm = "mlp" if (args.workload in (1, 2, 5) and os.path.exists(model)) else "cold"
    mlp = None
    if warm == "mlp":
        from paper_2607_17978_b300 import warmstart
        mlp, _ = warmstart.load(model, device=dev)
        plan.set_warm_start(mlp)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # > 126 MB L2

    def solve():
        return plan.solve(d_pos, d_spc, d_chi, d_J, qt, out=q_out, warm=("mlp" if warm == "mlp" else None))

    for _ in range(max(args.warmup, 1)):
        res = solve()
    torch.cuda.synchronize()
    launches0 = plan.query(0)["kernel_launches"]
    ev0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ev1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    iters, restarts = [], []
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    torch.cuda.profiler.start()                     # ncu --profile-from-start off captures the timed steps only
    for k in range(args.steps):
        flush.fill_(float(k))                       # evict the previous step's data from L2 (untimed)
        plan.stream.wait_stream(torch.cuda.current_stream(dev))
        ev0[k].record(plan.stream)
        res = solve()
        ev1[k].record(plan.stream)
        iters.append([i["iterations"] for i in res.info])
        restarts.append(max(i["restarts"] for i in res.info))
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    if world > 1:
        torch.distributed.barrier()
    clk = clocks.stop()
    t_steps = [a.elapsed_time(b) for a, b in zip(ev0, ev1)]
    ms = sum(t_steps) / len(t_steps)
    launches = (plan.query(0)["kernel_launches"] - launches0)
    ms = shard.max_over_ranks(ms, dev)          # the slowest rank sets the step time
    status = max(i["status"] for i in res.info)
    it_arr = np.array(iters, dtype=np.float64)               # steps x structures
    atoms_iters = float(np.mean(it_arr @ np.array([x.n for x in structs], dtype=np.float64)))
    it_mean = float(it_arr.mean())

    warm_used = min(i["warm_used"] for i in res.info) if warm == "mlp" else 0
    # ---- the same chosen form without the warm start (one solve): what the network gains
    cold_ms, cold_iters = None, None
    if warm == "mlp":
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(1.0)
        plan.stream.wait_stream(torch.cuda.current_stream(dev))
        a.record(plan.stream)
        rc = plan.solve(d_pos, d_spc, d_chi, d_J, qt, out=q_out)
        b.record(plan.stream)
        torch.cuda.synchronize()
        cold_ms = a.elapsed_time(b)
        cold_iters = float(np.mean([i["iterations"] for i in rc.info]))

    # ---- roofline of the dominant kernel (per-stage CUDA events on the plan's stream)
    prof = plan.profile_matvec(20)
    pairs_est = 0
    sb = stage_bytes(plan, args.precision, n_atoms, pairs_est)
    dom = max(prof, key=prof.get)
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6400.0
    achieved = sb[dom] / (prof[dom] * 1e-3) / 1e9
    traffic = load_traffic().get(f"{dom}:{args.workload}:{args.precision}")
    matvec_ms = sum(prof.values())
    matvec_bytes = sum(sb.values())

    # ---- plain FP64 GPU PCG (one structure per launch, no graph): the comparison denominator
    sample = list(range(0, n_struct, 16)) if n_struct > 1 else [0]
    plain_ms_sum, plain_iters, dq_plain = 0.0, [], 0.0
    offs = np.concatenate([[0], np.cumsum([x.n for x in structs])])
    for k in sample:
        s1 = structs[k]
        plain = qeq.plan_for_structures([s1], precision="fp64", graph=False, device=dev, **opts)
        a1 = [torch.tensor(v, device=dev) for v in qeq.pack([s1])[:4]]
        q1 = np.array([s1.q_tot])
        plain.solve(*a1, q1)
        torch.cuda.synchronize()
        n_plain = max(1, min(3, args.steps)) if n_struct == 1 else 1
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.fill_(0.0)
        plain.stream.wait_stream(torch.cuda.current_stream(dev))
        a.record(plain.stream)
        for _ in range(n_plain):
            rp = plain.solve(*a1, q1)
        b.record(plain.stream)
        torch.cuda.synchronize()
        plain_ms_sum += a.elapsed_time(b) / n_plain
        plain_iters.append(rp.info[0]["iterations"])
        dq_plain = max(dq_plain, float((q_out[offs[k]:offs[k + 1]] - rp.q).abs().max().item()))
        plain.close()
    plain_ms = plain_ms_sum * n_struct / len(sample)     # one structure after another, extrapolated

    # ---- end to end through the public API with pinned host buffers
    h_pos = torch.tensor(pos).pin_memory()
    h_spc = torch.tensor(spc).pin_memory()
    h_chi = torch.tensor(chi).pin_memory()
    h_J = torch.tensor(J).pin_memory()
    h_q = torch.empty(n_atoms, dtype=torch.float64).pin_memory()
    n_e2e = max(1, min(5, args.steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        d_pos.copy_(h_pos, non_blocking=True)
        d_spc.copy_(h_spc, non_blocking=True)
        d_chi.copy_(h_chi, non_blocking=True)
        d_J.copy_(h_J, non_blocking=True)
        r = solve()
        torch.cuda.current_stream(dev).wait_stream(plan.stream)
        h_q.copy_(q_out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = shard.max_over_ranks((time.perf_counter() - t0) / n_e2e, dev)
    atoms_iters_all = shard.sum_over_ranks(atoms_iters, dev) if sharded else world * atoms_iters
    h2d = int(pos.nbytes + spc.nbytes + chi.nbytes + J.nbytes)
    d2h = int(n_atoms * 8)

    if rank != 0:
        return 0
    cpu = None
    if world == 1 and not args.no_cpu_baseline:
        if n_struct > 1:
            v, cores, smp = cpu_oracle_dense_batch(structs)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": smp}
        else:
            t_mv, cores, reps = cpu_oracle_matvec_time(st)
            v = 1.0 / (t_mv * PCG_ITERS_REFERENCE)
            cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                   "sample": (f"FP64 Ewald matvec of the full {st.n}-atom cell by the CPU oracle (best of {reps}), "
                              f"x {PCG_ITERS_REFERENCE} PCG iterations: extrapolated to one solve")}
    value = n_total * 1000.0 / ms
    qi = plan.query(0)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "strong" if sharded else "weak",
        "vs_baseline": None, "dtype": "f32+f64" if args.precision == "mixed" else "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD_NAME[args.workload], "atoms": atoms_total, "structures": len(structs_all),
                   "mesh": list(qi["mesh"]) if n_struct == 1 else "per structure (autotuned)",
                   "spline_order": qi["spline_order"], "omega_A": round(qi["omega"], 4), "precision": args.precision,
                   "graph": True, "warm_start": warm, "preconditioner": args.precond, "charge_tol_e": 1e-5, "l2": "flushed between timed steps (256 MB write)",
                   "parallelism": f"sharded x{world}" if sharded else f"replicas x{world}"},
        "atoms_iters_per_s": atoms_iters_all / (ms * 1e-3),
        "pcg_iterations": it_mean, "pcg_restarts_max": int(max(restarts)), "status": status,
        "warm_start": {"kind": warm, "kept": bool(warm_used) if warm == "mlp" else None,
                       "cold_ms_per_step": cold_ms, "cold_pcg_iterations": cold_iters},
        "plain_fp64": {"value": n_struct * 1000.0 / plain_ms, "unit": UNIT, "ms_per_step": plain_ms,
                       "iterations": float(np.mean(plain_iters)), "speedup_of_chosen": plain_ms / ms,
                       "max_dq_vs_chosen_e": dq_plain,
                       "sample": ("every structure" if n_struct == 1 else
                                  f"{len(sample)} of {n_struct} structures (every 16th) solved one at a time, "
                                  f"time scaled by {n_struct}/{len(sample)}")},
        "matvec": {"ms": matvec_ms, "algorithmic_bytes": matvec_bytes,
                   "GBps": matvec_bytes / (matvec_ms * 1e-3) / 1e9,
                   "frac_hbm": matvec_bytes / (matvec_ms * 1e-3) / 1e9 / hbm,
                   "stages_ms": {k: round(v, 5) for k, v in prof.items()}},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_launch": sb[dom], "launch_ms": prof[dom]},
        "e2e": {"value": n_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    if cpu:
        line["cpu_baseline"] = cpu
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", type=int, default=2, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precond", default="fourier", choices=["fourier", "jacobi"],
                    help="preconditioner of the chosen form (the plain FP64 leg always uses Jacobi)")
    ap.add_argument("--warm", default="auto", choices=["auto", "mlp", "cold"],
                    help="learned warm start (auto: on for workloads 1, 2 and 5, the training recipe, when the model file exists)")
    ap.add_argument("--profile-cells", dest="cells", type=int, default=0,
                    help="profiling mode: solve a rock-salt cell of N^3 conventional cells only")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.cells > 0:
        return run_profile(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
