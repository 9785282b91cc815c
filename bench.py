"""Benchmark of the periodic QEq solve on one B300 (or N replicas).

One step = one complete cold- or warm-start QEq solve of the workload through
the C ABI (charges to 1e-5 e, final FP64 residual check included), inputs
resident on the device.  The default workload is the largest single-GPU cell,
the 980,000-atom rock-salt cell (50x50x50 conventional cells, 2% vacancies,
jitter 0.2 A, r_cut 8 A, ewald_tol 1e-6); the chosen form is mixed precision
(FP32 mesh, FP64 reductions), the Fourier-Woodbury preconditioner, the learned
warm start (rock-salt recipe) and the PCG iterations captured in CUDA graphs.
Beside it: the plain FP64 GPU PCG (Jacobi, no graph), the roofline of the
dominant matvec kernel (CUDA events on the plan's stream), the whole matvec
against the algorithmic byte model 24 S M + 28 N, the error of the chosen
form against the FP64 oracle (dense solve, or the oracle's residual on sampled
rows where a dense solve is infeasible), an end-to-end number through the
public API with host buffers, and the FP64 CPU oracle timed on the host cores.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload 5|1|2|3|4]

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
# Jacobi-PCG iterations of the plain FP64 solve at 1e-5 e, measured on the GPU with the
# current code (bench line "plain_fp64.iterations"), used by the reference arm to scale
# the CPU oracle's measured matvec time to a solve where the dense solve does not fit
# the time budget; the arm of ours uses the count measured in the same run.
PLAIN_PCG_ITERS = {1: 21, 2: 92, 3: 226, 5: 396}
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
def mesh_points(plan):
    """Sum over structures of S * M (species x mesh points): the real meshes of the byte model."""
    sm = 0
    for s in range(plan.n_struct):
        qi = plan.query(s)
        K = qi["mesh"]
        sm += K[0] * K[1] * K[2] * qi["n_species"]
    return sm


def stage_bytes(plan, prec: str, n_atoms: int):
    """Algorithmic DRAM bytes per launch of each matvec stage (all structures of the plan).

    The algorithmic model of one matvec is B = S M (4 spread write + 4 + 4 forward FFT
    + 4 + 4 inverse FFT + 4 gather read) + N (8 q + 12 pos + 8 y) = 24 S M + 28 N bytes
    in FP32 (mesh bytes doubled in FP64).  Per stage: the spread writes the mesh once and
    reads positions and charges (4 S M + 20 N), every FFT pass reads and writes the mesh
    once (8 S M; the passes beyond one per direction count against the matvec's
    efficiency, not against its budget), the gather reads the mesh once and writes y
    (4 S M + 8 N).  Real-space pair bytes are not part of the model.
    """
    rs = 4 if prec == "mixed" else 8           # one real mesh value
    SM = mesh_points(plan)
    return {
        "species_sums": n_atoms * (8 + 4),
        "spread": SM * rs + n_atoms * 20,
        "fft_z": 2 * SM * rs,
        "fft_y": 2 * SM * rs,
        "fft_x_green": 2 * SM * rs,
        "ifft_y": 2 * SM * rs,
        "ifft_z": 2 * SM * rs,
        "gather": SM * rs + n_atoms * 8,
    }


def matvec_model_bytes(plan, prec: str, n_atoms: int):
    """24 S M + 28 N (FP32; 48 S M + 28 N in FP64): the bytes one matvec must move."""
    rs = 4 if prec == "mixed" else 8
    return 6 * rs * mesh_points(plan) + 28 * n_atoms


def load_traffic():
    """DRAM traffic per launch of the dominant kernel from the committed ncu summary, if current."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        return json.load(open(path))
    except Exception:
        return {}


# ----------------------------------------------------------------------------- CPU oracle
def _cores():
    """All host cores for the CPU oracle's OpenMP loops (torchrun sets OMP_NUM_THREADS=1 in every
    rank, so the setting is overridden here and in the OpenMP runtime the oracle links)."""
    cores = len(os.sched_getaffinity(0))
    os.environ["OMP_NUM_THREADS"] = str(cores)
    try:
        import ctypes
        ctypes.CDLL("libgomp.so.1").omp_set_num_threads(cores)
    except OSError:
        pass
    return cores


def oracle_matvec_seconds(st, reps: int = 1):
    """Best wall time of the oracle's full FP64 Ewald matvec of ``st`` over ``reps`` calls."""
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    O.build_c()
    q = np.random.default_rng(0).normal(size=st.n)
    best = math.inf
    for _ in range(reps):
        t0 = time.perf_counter()
        O.ewald_matvec(st.cell, st.pos, st.sigma, q, k_e=synth.COULOMB_K_EV_A)
        best = min(best, time.perf_counter() - t0)
    return best


# full oracle matvecs above this many atoms do not fit the bench's CPU budget (minutes each):
# their time is extrapolated from two smaller cells of the same recipe
FULL_MATVEC_MAX_ATOMS = 200_000
SUBCELLS = (16, 24)          # conventional cells per edge of the two timed sub-cells


def oracle_matvec_estimate(workload: int, st, reps: int = 1):
    """Oracle FP64 matvec time of the workload cell: measured, or extrapolated by the power
    law t = a N^b through two timed sub-cells of the same recipe.  Returns (seconds, text)."""
    from paper_2607_17978_b300 import synth
    if st.n <= FULL_MATVEC_MAX_ATOMS:
        t = oracle_matvec_seconds(st, reps)
        return t, f"FP64 oracle Ewald matvec of the full {st.n}-atom cell: {t:.2f} s (measured)"
    sub = [synth.workload(workload, scale=k) for k in SUBCELLS]
    ts = [oracle_matvec_seconds(x, reps) for x in sub]
    b = math.log(ts[1] / ts[0]) / math.log(sub[1].n / sub[0].n)
    t = ts[1] * (st.n / sub[1].n) ** b
    return t, (f"FP64 oracle Ewald matvec measured on {sub[0].n} and {sub[1].n}-atom cells of the same recipe "
               f"({ts[0]:.2f} s, {ts[1]:.2f} s), extrapolated to {st.n} atoms by t ~ N^{b:.2f}: {t:.1f} s")


def oracle_error_single(workload: int, st, q, mu, n_rows: int = 64):
    """Error of GPU charges q (input order) against the FP64 oracle.

    Dense bordered solve up to 2,000 atoms (max |q - q*|); the oracle's full matvec up to
    FULL_MATVEC_MAX_ATOMS (projected residual P(A q + chi) on every atom and the certified
    bound ||q - q*||_2 <= ||P(A q + chi)||_2 / J_min); above, the residual on n_rows seeded
    sampled rows.  Returns (dict, seconds spent)."""
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    O.build_c()
    KE = synth.COULOMB_K_EV_A
    t0 = time.perf_counter()
    if st.n <= 2000:
        sol = O.solve_structure(st, k_e=KE)
        out = {"kind": "dense bordered oracle solve, every atom", "max_dq_e": float(np.abs(q - sol.q).max()),
               "dmu_eV": float(abs(mu - sol.mu))}
    elif st.n <= FULL_MATVEC_MAX_ATOMS:
        y = O.ewald_matvec(st.cell, st.pos, st.sigma, q, k_e=KE)
        Pr, mu_o = O.projected_residual(y, st.J, st.chi, q)
        out = {"kind": "oracle FP64 matvec of the chosen charges, every atom",
               "residual_inf_eV": float(np.abs(Pr).max()), "bound_l2_e": O.certified_bound(Pr, st.J),
               "dmu_eV": float(abs(mu - mu_o)), "stop_threshold_eV": 0.5 * 1e-5 * float(st.J.min())}
    else:
        rows = np.sort(np.random.default_rng(workload).choice(st.n, n_rows, replace=False))
        omega = 11.0
        y = O.ewald_matvec(st.cell, st.pos, st.sigma, q, k_e=KE, omega=omega, rows=rows)
        r = y + st.J[rows] * q[rows] + st.chi[rows] - mu
        out = {"kind": f"oracle FP64 residual (A q + chi - mu) of the chosen charges on {n_rows} seeded sampled rows",
               "residual_inf_eV": float(np.abs(r).max()), "stop_threshold_eV": 0.5 * 1e-5 * float(st.J.min())}
    return out, time.perf_counter() - t0


def oracle_error_batch(structs, q, mu, every: int = 64):
    """Dense oracle solves of every ``every``-th structure of a batch: max |q - q*|, and their time."""
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    O.build_c()
    off = np.concatenate([[0], np.cumsum([x.n for x in structs])])
    sample = list(range(0, len(structs), every))
    worst, dmu = 0.0, 0.0
    t0 = time.perf_counter()
    for k in sample:
        sol = O.solve_structure(structs[k], k_e=synth.COULOMB_K_EV_A)
        worst = max(worst, float(np.abs(q[off[k]:off[k + 1]] - sol.q).max()))
        dmu = max(dmu, float(abs(mu[k] - sol.mu)))
    t = time.perf_counter() - t0
    return ({"kind": f"dense bordered oracle solves of {len(sample)} of {len(structs)} structures (every {every}th)",
             "max_dq_e": worst, "dmu_eV": dmu}, len(sample) / t, t)


def charge_training_leg(dev, flush, n_struct: int = 256, steps: int = 3, precision: str = "mixed"):
    """4G charge training on cached dense matrices (qeq_dense_*): E of a fixed synthetic
    training batch assembled once, then per step a re-inversion with a new (learned) hardness,
    the charges and their backward pass.  Roofline of the inversion kernel against the FP64
    rate (FP64 arithmetic bound)."""
    import torch
    from paper_2607_17978_b300 import qeq, synth
    structs = synth.training_structures(n_struct, cfg_id=6, first=0, n_min=64, n_max=512)
    ns = [x.n for x in structs]
    pos, spc, chi, J, qt = qeq.pack(structs)
    d_pos, d_spc = torch.tensor(pos, device=dev), torch.tensor(spc, device=dev)
    d_chi, d_J = torch.tensor(chi, device=dev), torch.tensor(J, device=dev)
    dense = qeq.dense_for_structures(structs, device=dev, precision=precision)
    rng = np.random.default_rng(1)
    Js = [d_J * torch.tensor(rng.uniform(0.9, 1.1, len(J)), device=dev) for _ in range(steps + 1)]
    gq = torch.tensor(rng.normal(size=len(J)), device=dev)

    def ev():
        return torch.cuda.Event(enable_timing=True)

    torch.cuda.synchronize()
    a, b = ev(), ev()
    dense.stream.wait_stream(torch.cuda.current_stream(dev))
    a.record(dense.stream)
    dense.assemble(d_pos, d_spc)
    b.record(dense.stream)
    torch.cuda.synchronize()
    assemble_ms = a.elapsed_time(b)
    dense.invert(Js[0])
    q, _ = dense.charges(d_chi, qt)
    dense.backward(q, gq)
    torch.cuda.synchronize()
    step_ms, inv_ms = [], []
    for k in range(1, steps + 1):
        flush.fill_(3.0)
        e0, e1, e2 = ev(), ev(), ev()
        dense.stream.wait_stream(torch.cuda.current_stream(dev))
        e0.record(dense.stream)
        dense.invert(Js[k])
        e1.record(dense.stream)
        q, _ = dense.charges(d_chi, qt)
        dense.backward(q, gq)
        e2.record(dense.stream)
        torch.cuda.synchronize()
        step_ms.append(e0.elapsed_time(e2))
        inv_ms.append(e0.elapsed_time(e1))
    launches = dense.query(0)["kernel_launches"]
    dense.close()
    # operations of the inversion per structure: Cholesky n^3/3, triangular inverse n^3/3,
    # U^-1 U^-T n^3/3 (multiply and add counted apart), the border O(n^2).  Peaks: FP64 1.25
    # TFLOP/s nominal; FP32 148 SMs x 128 lanes x 2 FLOP x 2.032 GHz = 77.0 TFLOP/s
    flops = float(sum(float(n) ** 3 for n in ns))
    t_inv = statistics.median(inv_ms) * 1e-3
    peak = 77.0 if precision == "mixed" else 1.25
    return {"structures": len(structs), "atoms": int(sum(ns)), "atoms_per_structure": [min(ns), max(ns)],
            "recipe": "rock-salt training cells (jitter 0.2 A, 2% vacancies), log-uniform 64-512 atoms",
            "assemble_ms": assemble_ms, "step_ms": statistics.median(step_ms),
            "structures_per_s": len(structs) / (statistics.median(step_ms) * 1e-3),
            "step": "re-invert with a new hardness + charges + backward (dL/dchi, dL/dJ)",
            "precision": ("FP32 inverse, charges and gradients refined to FP64 (2 steps)" if precision == "mixed"
                          else "FP64 inverse"),
            "invert_ms": statistics.median(inv_ms), "kernel_launches_total": int(launches),
            "roofline": {"kernel": "k_dense_invert", "bound": "alu", "achieved": flops / t_inv / 1e12,
                         "peak": peak, "unit": "TFLOP/s (%s)" % ("FP32" if precision == "mixed" else "FP64"),
                         "frac": flops / t_inv / 1e12 / peak,
                         "peak_source": ("FP32 CUDA-core rate from unit counts and the 2032 MHz clock"
                                         if precision == "mixed" else "nominal FP64 rate of this part"),
                         "flops_per_launch": flops}}


def run_reference(args):
    """The CPU oracle as it stands, timed on the host cores on this workload."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    from oracle import qeq_oracle as O
    from paper_2607_17978_b300 import synth
    structs = workload_structs(args.workload)
    cores = _cores()
    O.build_c()
    extra = {}
    if len(structs) > 1:
        # one dense bordered solve per step, cycling through every 64th structure
        sample = list(range(0, len(structs), 64))
        for k in range(args.warmup):
            O.solve_structure(structs[sample[k % len(sample)]], k_e=synth.COULOMB_K_EV_A)
        t0 = time.perf_counter()
        for k in range(args.steps):
            O.solve_structure(structs[sample[k % len(sample)]], k_e=synth.COULOMB_K_EV_A)
        step_s = (time.perf_counter() - t0) / args.steps
        solve_s = step_s
        desc = (f"dense FP64 oracle solve (Ewald assembly + bordered LU) of one structure per step, cycling through "
                f"every 64th of the {len(structs)} structures")
        atoms = sum(x.n for x in structs)
    elif structs[0].n <= 2000:
        st = structs[0]
        for _ in range(args.warmup):
            O.solve_structure(st, k_e=synth.COULOMB_K_EV_A)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            O.solve_structure(st, k_e=synth.COULOMB_K_EV_A)
        step_s = solve_s = (time.perf_counter() - t0) / args.steps
        desc = f"dense FP64 oracle solve (Ewald assembly + bordered LU) of the {st.n}-atom cell per step"
        atoms = st.n
    else:
        # one oracle FP64 matvec per step (of the cell itself when it fits, else of a sub-cell of
        # the same recipe, alternating the two sizes of the extrapolation); a solve is that
        # matvec time x the plain-PCG iteration count of this workload
        st = structs[0]
        iters = PLAIN_PCG_ITERS[args.workload]
        cells = [st] if st.n <= FULL_MATVEC_MAX_ATOMS else [synth.workload(args.workload, scale=k) for k in SUBCELLS]
        for k in range(args.warmup):
            oracle_matvec_seconds(cells[k % len(cells)])
        ts = [[] for _ in cells]
        t0 = time.perf_counter()
        for k in range(args.steps):
            ts[k % len(cells)].append(oracle_matvec_seconds(cells[k % len(cells)]))
        step_s = (time.perf_counter() - t0) / args.steps
        for k, x in enumerate(ts):  # fewer steps than sub-cells: time the missing ones once, untimed
            if not x:
                x.append(oracle_matvec_seconds(cells[k]))
        if len(cells) == 1:
            t_mv = float(np.mean(ts[0]))
            how = f"measured, mean of {len(ts[0])}"
        else:
            m = [float(np.mean(x)) for x in ts]
            b = math.log(m[1] / m[0]) / math.log(cells[1].n / cells[0].n)
            t_mv = m[1] * (st.n / cells[1].n) ** b
            how = (f"steps alternate {cells[0].n}- and {cells[1].n}-atom cells of the same recipe "
                   f"({m[0]:.2f} s, {m[1]:.2f} s), extrapolated to {st.n} atoms by t ~ N^{b:.2f}")
        solve_s = t_mv * iters
        desc = (f"one FP64 oracle Ewald matvec per step ({how}); solve = matvec {t_mv:.2f} s x {iters} plain "
                f"Jacobi-PCG iterations (measured on the GPU for this workload)")
        extra = {"solve_seconds_extrapolated": solve_s, "matvec_seconds": t_mv}
        atoms = st.n
    value = 1.0 / solve_s
    line = {"metric": METRIC, "value": value, "unit": UNIT, "impl": "reference", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD_NAME[args.workload], "atoms": atoms, "structures": len(structs)},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "sample": desc},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    line.update(extra)
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
    plan = qeq.plan_for_structures([st], precision=args.precision, ewald_tol=1e-6, r_cut=8.0, graph=not args.no_graph)
    pos, spc, chi, J, qt = qeq.pack([st])
    d = [torch.tensor(a, device="cuda") for a in (pos, spc, chi, J)]
    torch.cuda.profiler.start()                     # ncu --profile-from-start off: the solves ...
    for _ in range(args.steps):
        r = plan.solve(*d, qt)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    stages = plan.profile_matvec(5)
    # ... and, with --forces, one force-trick evaluation (lambda from a second solve, forces, stress)
    extra = {}
    if args.forces:
        dEdq = plan.matvec(d[0], d[1], r.q, fp64=True)
        lam = plan.solve(d[0], d[1], dEdq, d[3], np.zeros(1)).q
        plan.forces(d[0], d[1], r.q, lam)
        plan.stress(d[0], d[1], r.q, lam)
        torch.cuda.synchronize()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        torch.cuda.profiler.start()
        plan.stream.wait_stream(torch.cuda.current_stream())
        ev[0].record(plan.stream)
        plan.forces(d[0], d[1], r.q, lam)
        ev[1].record(plan.stream)
        plan.stress(d[0], d[1], r.q, lam)
        ev[2].record(plan.stream)
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        extra = {"forces_ms": ev[0].elapsed_time(ev[1]), "stress_ms": ev[1].elapsed_time(ev[2])}
    print(json.dumps({"profile_case": f"rocksalt {args.cells}^3", "atoms": st.n, "mesh": plan.query(0)["mesh"],
                      "iterations": r.info[0]["iterations"], "stages_ms": stages, **extra}))
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
    plan = qeq.plan_for_structures(structs, precision=args.precision, device=dev, preconditioner=args.precond,
                                   graph=not args.no_graph, **opts)
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
    sb = stage_bytes(plan, args.precision, n_atoms)
    dom = max(prof, key=prof.get)
    pk = peaks()
    hbm = pk.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or 6400.0
    achieved = sb[dom] / (prof[dom] * 1e-3) / 1e9
    traffic = load_traffic().get(f"{dom}:{args.workload}:{args.precision}")
    matvec_ms = sum(prof.values())
    matvec_bytes = matvec_model_bytes(plan, args.precision, n_atoms)

    # ---- force trick (SI eq. 4g_force_trick) after the solve: dE/dq = E q (FP64 matvec, no
    # hardness), lambda from a second solve (chi := dE/dq, q_tot = 0), then qeq_forces(q, lambda)
    zeros = np.zeros(n_struct)
    box = {}

    def trick():
        # dE/dq = E q only feeds the lambda solve's right-hand side: the plan's precision will do
        box["dEdq"] = plan.matvec(d_pos, d_spc, q_out, fp64=(args.precision == "fp64"))
        box["lam"] = plan.solve(d_pos, d_spc, box["dEdq"], d_J, zeros)
        box["F"] = plan.forces(d_pos, d_spc, q_out, box["lam"].q)

    def timed(fn, n=3):
        fn()
        torch.cuda.synchronize()
        tot = 0.0
        for _ in range(n):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            flush.fill_(2.0)
            plan.stream.wait_stream(torch.cuda.current_stream(dev))
            a.record(plan.stream)
            fn()
            b.record(plan.stream)
            torch.cuda.synchronize()
            tot += a.elapsed_time(b)
        return tot / n

    trick_ms = timed(trick)
    lam_q = box["lam"].q
    trick_parts = {
        "dEdq_matvec_ms": timed(lambda: plan.matvec(d_pos, d_spc, q_out, fp64=(args.precision == "fp64"))),
        "lambda_solve_ms": timed(lambda: plan.solve(d_pos, d_spc, box["dEdq"], d_J, zeros)),
        "forces_ms": timed(lambda: plan.forces(d_pos, d_spc, q_out, lam_q)),
        "forces_without_lambda_ms": timed(lambda: plan.forces(d_pos, d_spc, q_out)),
        "stress_ms": timed(lambda: plan.stress(d_pos, d_spc, q_out, lam_q)),
    }
    trick_iters = float(np.mean([i["iterations"] for i in box["lam"].info]))

    # ---- the two-RHS formulation (plain PCG on A t = 1 and A s = -chi, no constraint), cold, in
    # the chosen precision and preconditioner: the solver variant the paper compares against
    two = qeq.plan_for_structures(structs, precision=args.precision, device=dev, preconditioner=args.precond,
                                  graph=not args.no_graph, solver="two_rhs", **opts)
    two.solve(d_pos, d_spc, d_chi, d_J, qt)
    torch.cuda.synchronize()
    a2, b2 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    flush.fill_(4.0)
    two.stream.wait_stream(torch.cuda.current_stream(dev))
    a2.record(two.stream)
    r2 = two.solve(d_pos, d_spc, d_chi, d_J, qt)
    b2.record(two.stream)
    torch.cuda.synchronize()
    two_rhs = {"ms_per_step": a2.elapsed_time(b2), "value": n_struct * 1000.0 / a2.elapsed_time(b2),
               "unit": UNIT, "pcg_iterations": float(np.mean([i["iterations"] for i in r2.info])),
               "max_dq_vs_chosen_e": float((r2.q - q_out).abs().max().item()),
               "form": "cold start, two unconstrained PCG solves, same precision and preconditioner"}
    two.close()

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
        n_plain = max(1, min(3, args.steps)) if (n_struct == 1 and s1.n < 100_000) else 1
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
    # ---- error of the chosen form against the FP64 oracle, and the oracle timed on the host cores
    cpu, oracle_err = None, None
    if not args.no_oracle:
        cores = _cores()
        q_np = q_out.cpu().numpy()
        mu_np = res.mu.cpu().numpy()
        if n_struct > 1:
            oracle_err, v, t_or = oracle_error_batch(structs, q_np, mu_np)
            if world == 1:
                cpu = {"value": v, "unit": UNIT, "cores": cores, "kind": "oracle",
                       "sample": f"{oracle_err['kind']}: {t_or:.1f} s (the same solves that give the oracle error)"}
        else:
            oracle_err, t_or = oracle_error_single(args.workload, st, q_np, float(mu_np[0]))
            if world == 1:
                if st.n <= 2000:
                    t_solve = t_or
                    cpu = {"value": 1.0 / t_solve, "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"dense FP64 oracle solve (Ewald assembly + bordered LU) of the cell: {t_solve:.3f} s"}
                else:
                    it_p = float(np.mean(plain_iters))
                    t_mv, how = oracle_matvec_estimate(args.workload, st)
                    cpu = {"value": 1.0 / (t_mv * it_p), "unit": UNIT, "cores": cores, "kind": "oracle",
                           "sample": f"{how}; x {it_p:.0f} plain Jacobi-PCG iterations measured in this run = one solve"}
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
                   "graph": not args.no_graph, "warm_start": warm, "preconditioner": args.precond, "charge_tol_e": 1e-5, "l2": "flushed between timed steps (256 MB write)",
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
        "matvec": {"ms": matvec_ms, "model": "24 S M + 28 N bytes (FP32 mesh; 48 S M + 28 N in FP64)",
                   "algorithmic_bytes": matvec_bytes,
                   "GBps": matvec_bytes / (matvec_ms * 1e-3) / 1e9,
                   "frac_hbm": matvec_bytes / (matvec_ms * 1e-3) / 1e9 / hbm,
                   "stages_ms": {k: round(v, 5) for k, v in prof.items()},
                   "stage_frac_hbm": {k: round(sb[k] / (prof[k] * 1e-3) / 1e9 / hbm, 4) for k in prof if prof[k] > 0}},
        "roofline": {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic, "peak_source": f"{peak_src} (MEASURED_PEAKS.json hbm_gbs)",
                     "algorithmic_bytes_per_launch": sb[dom], "launch_ms": prof[dom]},
        "e2e": {"value": n_total / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "clocks": clk,
    }
    line["two_rhs_solver"] = two_rhs
    line["force_trick"] = {
        "ms_per_step": trick_ms, "atoms_per_s": n_atoms / (trick_ms * 1e-3),
        "lambda_pcg_iterations": trick_iters, "vs_charge_solve": trick_ms / ms,
        "parts_ms": {k: round(v, 4) for k, v in trick_parts.items()},
        "form": ("potential meshes in the plan's precision (%s), pair derivative and sums in FP64; "
                 "stress in FP64; lambda solve in the chosen form, cold start" % args.precision),
    }
    if rank == 0:
        line["charge_training"] = charge_training_leg(dev, flush, precision="mixed")
        line["charge_training"]["fp64_inverse"] = {
            k: v for k, v in charge_training_leg(dev, flush, precision="fp64").items()
            if k in ("step_ms", "structures_per_s", "invert_ms", "roofline")}
    if oracle_err:
        line["oracle_error"] = oracle_err
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
    ap.add_argument("--workload", type=int, default=5, choices=[1, 2, 3, 4, 5])
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--no-oracle", action="store_true",
                    help="skip the oracle error and the CPU oracle baseline (host work after the GPU legs)")
    ap.add_argument("--precond", default="fourier", choices=["fourier", "jacobi"],
                    help="preconditioner of the chosen form (the plain FP64 leg always uses Jacobi)")
    ap.add_argument("--warm", default="auto", choices=["auto", "mlp", "cold"],
                    help="learned warm start (auto: on for workloads 1, 2 and 5, the training recipe, when the model file exists)")
    ap.add_argument("--no-graph", action="store_true",
                    help="host-paced PCG rounds instead of the device-paced graph (same kernels; for ncu, which "
                         "cannot profile the kernel nodes of a graph with conditional nodes)")
    ap.add_argument("--forces", action="store_true",
                    help="with --profile-cells: also one force-trick evaluation (forces and stress)")
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
