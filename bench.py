#!/usr/bin/env python
"""Benchmark of the CheFSI SCF hot path on GB300.

Metric: seconds until the SCF free energy is within 1e-5 Ha/atom of the FP64 CPU oracle's
converged value and stays there (mixed precision: FP32 Chebyshev filter, FP64 subspace
eigensolve and reductions).  One step = one complete SCF of the workload cell from the SAD guess
and seeded orbitals already resident on the device (all hot-path rows: Poisson/XC, filter,
Rayleigh-Ritz, occupations, density, mixing, energy, final FP64 pass, forces).

Default workload: 64 synthetic atoms on a 4x4x4 lattice (edge 20.52 bohr, 80^3 grid, 154 states,
degree-20 filter), the shape of the paper's O(100-500)-atom Gamma-point LDA runs.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

With N > 1 (torchrun) each rank solves its own replica (the method does not shard this cell).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "SCF s-to-1e-5 Ha/atom, mixed+learned vs FP64 GPU; H\u00b7X stencil % of HBM peak"
UNIT = "s"
TOL_PER_ATOM = 1e-5


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=3)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--workload", default="lattice64_80")
    p.add_argument("--precision", choices=["mixed", "fp64"], default="mixed")
    p.add_argument("--cpu-sample-seconds", type=float, default=20.0)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-fp64-compare", action="store_true")
    return p.parse_args()


def cell_for(name):
    import workloads
    return {"lattice64_80": workloads.lattice64_cell, "two_atom_24": workloads.two_atom_cell,
            "lattice216_120": workloads.lattice216_cell}[name]()


def golden(name):
    """The oracle's converged reference for the workload (tests/golden/make_golden.py), or None."""
    path = os.path.join(ROOT, "tests", "golden", name + ".json")
    if not os.path.exists(path):
        return None
    return json.load(open(path))


def hit_time(log, e_ref, natom):
    """First time after which |F - F_ref|/natom <= tol holds for every later iteration."""
    t = None
    for rec in log:
        ok = abs(rec["energy"] - e_ref) / natom <= TOL_PER_ATOM
        if ok and t is None:
            t = rec["seconds"]
        elif not ok:
            t = None
    return t


class ClockSampler:
    """nvidia-smi clocks / throttle reasons of this process's GPU, sampled every 200 ms."""

    FIELDS = ("uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) == 8 and (self.uuid is None or parts[0] == self.uuid):
                self.rows.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4) if r[4 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def stencil_source_hash():
    h = hashlib.sha256()
    for f in ("stencil_impl.cuh", "stencil_f32.cu"):
        h.update(open(os.path.join(ROOT, "paper_2005_10431_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(workload, variant):
    """Per-launch DRAM traffic (read + write) of the stencil tile `variant` from the committed ncu
    capture (profiles/stencil_traffic.json), if it was taken on the current kernel source; else None."""
    p = os.path.join(ROOT, "profiles", "stencil_traffic.json")
    if not os.path.exists(p):
        return None
    e = json.load(open(p)).get(workload, {}).get(variant)
    if not e or e.get("source_hash") != stencil_source_hash():
        return None
    return e


# ---------------------------------------------------------------------------------------
# CPU baseline: the FP64 oracle as it stands, on a bounded sample of the same workload
# ---------------------------------------------------------------------------------------
_ORACLE_CACHE = {}


def oracle_sample(name, budget_s):
    """Time full-block oracle H X applications on the workload (bounded), and scale to the metric:
    the oracle's own SCF needs (passes x (degree + 1)) block applications of H until its energy is
    within 1e-5 Ha/atom of its converged value (4 passes in the first iteration, then 1)."""
    import numpy as np
    import workloads
    from oracle import ham, scf as oscf
    if name not in _ORACLE_CACHE:
        cell = cell_for(name)
        _ORACLE_CACHE[name] = (cell, oscf.Problem(cell), workloads.initial_orbitals(cell.seed, cell.ngrid, cell.nstates))
    cell, pr, X = _ORACLE_CACHE[name]
    g = golden(name)
    V = np.full(cell.ngrid, -0.3)
    times = []
    t_start = time.time()
    while True:
        t0 = time.time()
        ham.apply_h(cell, X, V, pr.P[0], pr.E)
        times.append(time.time() - t0)
        if time.time() - t_start > budget_s or len(times) >= 3:
            break
    t_hx = min(times)
    i_hit = None
    if g is not None:
        hist = g["history"]
        e_ref = g["energy"]
        for rec in hist:
            ok = abs(rec["energy"] - e_ref) / cell.natom <= TOL_PER_ATOM
            if ok and i_hit is None:
                i_hit = rec["iter"]
            elif not ok:
                i_hit = None
        passes = 4 + (i_hit if i_hit is not None else len(hist))
    else:
        passes = 4 + 40   # no oracle run recorded: an assumed 40 SCF iterations
    n_hx = passes * (cell.cheb_degree + 1)
    threads = os.cpu_count() or 1
    return {"value": t_hx * n_hx, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": (f"{len(times)} full-block FP64 oracle H.X applications ({cell.ngrid} points x {cell.nstates} "
                       f"states, best {t_hx:.2f} s) scaled by the {n_hx} block applications the oracle SCF used to "
                       f"reach 1e-5 Ha/atom ({passes} CheFSI passes of degree {cell.cheb_degree} + RR)")}


# ---------------------------------------------------------------------------------------
def max_over_ranks(dist, vals, device):
    """Element-wise maximum of a list of floats over all ranks (the slowest replica sets the time)."""
    import torch
    t = torch.tensor([float(v) for v in vals], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(x) for x in t.tolist()]


def run_reference(args, rank, world):
    if rank != 0:
        return
    cpu = oracle_sample(args.workload, args.cpu_sample_seconds)
    steps = []
    for _ in range(args.warmup + args.steps):
        steps.append(oracle_sample(args.workload, 1.0)["value"])
    vals = steps[args.warmup:]
    v = statistics.mean(vals)
    cpu_line = dict(cpu, value=v)
    out = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1e3 * v, "higher_is_better": False, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": args.workload, "l2": "inputs larger than L2"},
           "impl": "reference", "cpu_baseline": cpu_line,
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


def run_ours(args, rank, world, dist):
    import numpy as np
    import torch
    import paper_2005_10431_gb300 as sd

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    cell = cell_for(args.workload)
    g = golden(args.workload)
    # without the oracle's converged energy the time-to-tolerance cannot be measured (value null)
    e_ref = g["energy"] if g else float("nan")
    prec = sd.SDFT_MIXED if args.precision == "mixed" else sd.SDFT_FP64
    # the metric is the time until the energy settles within 1e-5 Ha/atom of the oracle (about 30
    # iterations here), so each step stops after 100 iterations even where the density tolerance
    # is not yet met
    opts = dict(nstates=cell.nstates, cheb_degree=cell.cheb_degree, precision=prec, scf_tol=cell.scf_tol,
                max_scf=100, final_fp64_pass=1 if prec == sd.SDFT_MIXED else 0, kT=cell.kT, seed=cell.seed)
    stream = torch.cuda.Stream()
    ctx = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, opts, stream=stream)

    def one_step():
        sd.sdft_reset(ctx)
        r = sd.sdft_scf(ctx)
        log = sd.sdft_get_scf_log(ctx)
        return r, log

    for _ in range(args.warmup):
        one_step()
    sd.sdft_set_timing(ctx, True)
    sd.sdft_reset_kernel_stats(ctx)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    n0 = sd.sdft_launch_count(ctx)
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hits, niters, energies, converged = [], [], [], []
    with ClockSampler(uuid) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            r, log = one_step()
            hits.append(hit_time(log, e_ref, cell.natom))
            niters.append(r["niter"])
            energies.append(r["energy"])
            converged.append(bool(r["converged"]))
        ev1.record(stream)
        torch.cuda.synchronize()
    if dist:
        dist.barrier()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    launches = sd.sdft_launch_count(ctx) - n0
    stats = sd.sdft_get_kernel_stats(ctx)
    sd.sdft_set_timing(ctx, False)
    ok_hits = [h for h in hits if h is not None]
    value = statistics.mean(ok_hits) if len(ok_hits) == len(hits) else float("nan")
    ms_per_step = 1e3 * elapsed / args.steps
    if dist:
        value, ms_per_step = max_over_ranks(dist, [value if value == value else 1e30, ms_per_step], "cuda")
        value = float("nan") if value >= 1e30 else value
    if value != value:
        value = None   # some step never settled within the tolerance of the oracle energy
    # roofline of the dominant kernel (stencil + Chebyshev step)
    st = stats["stencil"]
    peak, peak_kind = measured_peaks()
    achieved = st["bytes"] / st["seconds"] / 1e9 if st["seconds"] > 0 else 0.0
    per_launch_bytes = st["bytes"] / max(1, st["launches"])
    vidx, vname = sd.sdft_get_stencil_variant(ctx, False)
    rec = recorded_traffic(args.workload, vname)
    # the capture is one launch with Yprev; scale its DRAM bytes to the average launch of this run
    traffic = (rec["dram_bytes_per_launch"] * (st["bytes"] / max(1, st["launches"])) / rec["algorithmic_bytes"]
               if rec else None)
    kname = ("cheb_row_kernel" if vname.startswith("row") else "cheb_step_kernel") + f" [{vname}]"
    roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
            "traffic": traffic, "kernel": kname + " (fused stencil H.Y + Chebyshev 3-term update)",
            "algorithmic_bytes_per_launch": per_launch_bytes, "avg_launch_ms": 1e3 * st["seconds"] / max(1, st["launches"]),
            "peak_source": f"{peak_kind} hbm_gbs", "apps_per_s": achieved * 1e9 / 12.0}
    # end to end through the C ABI with host inputs: create (H2D) + SCF + D2H of results
    e2e_vals = []
    h2d = cell.pos.nbytes + cell.natom * 4 + 6 * 8 * len(cell.species)
    d2h = (cell.nstates * 8 * 2) + cell.ngrid * 8 + cell.natom * 3 * 8
    for _ in range(max(1, min(args.steps, 2))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        c2 = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, opts, stream=stream)
        r = sd.sdft_scf(c2)
        log = sd.sdft_get_scf_log(c2)
        eig = sd.sdft_get_eigenvalues(c2)
        rho = sd.sdft_get_density(c2)
        f = sd.sdft_get_forces(c2)
        t1 = time.perf_counter()
        sd.sdft_destroy(c2)
        h = hit_time(log, e_ref, cell.natom)
        e2e_vals.append((t1 - t0) - (r["t_total"] - h) if h is not None else None)
        del eig, rho, f
    clocks = clk.summary()
    # the same SCF started from the learned density (network trained on the 64-atom sequence)
    learned = None
    wpath = os.path.join(ROOT, "paper_2005_10431_gb300", "weights", "mlp_qmd64.npy")
    if os.path.exists(wpath) and cell.ngrid == 80 ** 3:
        params = torch.from_numpy(np.load(wpath).astype(np.float32)).cuda()
        sd.sdft_reset(ctx)
        sd.sdft_mlp_predict(ctx, params)
        rl = sd.sdft_scf(ctx)
        logl = sd.sdft_get_scf_log(ctx)
        hl = hit_time(logl, e_ref, cell.natom)
        learned = {"hit_s": hl, "niter": rl["niter"], "energy": rl["energy"],
                   "dE_per_atom": abs(rl["energy"] - e_ref) / cell.natom if g else None}
    # the plain FP64 GPU SCF on the same cell, for the mixed-vs-FP64 comparison of the metric
    fp64 = None
    if not args.no_fp64_compare and prec == sd.SDFT_MIXED:
        o64 = dict(opts, precision=sd.SDFT_FP64, final_fp64_pass=0)
        c64 = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, dict(o64, max_scf=2), stream=stream)
        sd.sdft_scf(c64)                      # warm-up: library/solver initialisation
        sd.sdft_destroy(c64)
        c64 = sd.sdft_create(cell.L, cell.n, cell.pos, cell.types, cell.species, o64, stream=stream)
        r64 = sd.sdft_scf(c64)
        log64 = sd.sdft_get_scf_log(c64)
        h64 = hit_time(log64, e_ref, cell.natom)
        fp64 = {"hit_s": h64, "niter": r64["niter"], "energy": r64["energy"], "converged": bool(r64["converged"]),
                "s_per_iter": log64[-1]["seconds"] / max(1, len(log64)),
                "speedup_mixed_vs_fp64": (h64 / value) if (h64 and value) else None}
        sd.sdft_destroy(c64)
    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if prec == sd.SDFT_MIXED else "f64", "data": "synthetic",
        "config": {"workload": args.workload, "natom": cell.natom, "grid": list(cell.n), "nstates": cell.nstates,
                   "cheb_degree": cell.cheb_degree, "l2": "inputs larger than L2 (315 MB blocks)",
                   "parallelism": f"replicas{world}"},
        "roofline": roof,
        "e2e": {"value": statistics.mean(e2e_vals) if all(v is not None for v in e2e_vals) else None,
                "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clocks,
        "scf": {"niter": niters, "energy": energies, "oracle_energy": e_ref if g else None, "converged": converged,
                "hit_s": hits, "dE_per_atom": [abs(e - e_ref) / cell.natom for e in energies] if g else None},
        "kernel_seconds": {k: v["seconds"] for k, v in stats.items()},
        "fp64_gpu": fp64,
        "learned_guess": learned,
    }
    if g is None:
        out["value"] = None
        out["reference"] = f"oracle reference tests/golden/{args.workload}.json missing"
    if rank == 0 and not args.no_cpu_baseline and g is not None:
        out["cpu_baseline"] = oracle_sample(args.workload, args.cpu_sample_seconds)
    if rank == 0:
        print(json.dumps(out, allow_nan=False), flush=True)
    sd.sdft_destroy(ctx)


def main():
    args = parse()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    dist = None
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() and args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, dist)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
