"""Benchmark of the SLRF hot path (enhanced ParaSLRF, Alg. 2) on one GB300.

One step = one slrf_solve of the workload: every outer iteration's filter apply (all
poles x columns by COCG), B-orthogonalisation against the locked vectors, Cholesky-QR2,
Rayleigh-Ritz, residuals, locking and the warm start.  Default workload: the 3D Q1
linear-elasticity box on 64 x 64 x 32 nodes (3 dof per node, the z = 0 layer clamped,
n = 380,928, 29.6M stored entries, lognormal Young's modulus), gamma = 220.8176 (305
eigenpairs below it), block 480, m = 8 poles, Jacobi-preconditioned inner solves, complex-FP32
COCG in FP64 refinement (It_max 23); the same solve in FP64 is the "compare" record.  Other
workloads (--workload): q1_lap_41 (3D Q1 Laplacian on 41^3 nodes), elast_32 / elast_48,
bar1d_2000, batch64 (64 uneven pencils solved together), sens48 (48 scaled pencils).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun each rank solves its own copy (independent problems: weak scaling, no
collective on the data path); rank 0 prints one JSON line.
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

METRIC = "eigenpairs/s and shifted column-solves/s at resid\u22641e-8; SpMM HBM GB/s vs peak"
# Derived ALU peaks of GB300 (152 SMs at 2.07 GHz): FP64 2 FMA/clock/SM (measured 1.197 TFLOP/s
# at 1.98 GHz), FP32 128 FMA/clock/SM.
FP64_PEAK_TFLOPS = 152 * 2 * 2 * 2.07e9 / 1e12
FP32_PEAK_TFLOPS = 152 * 128 * 2 * 2.07e9 / 1e12
DEFAULT_WORKLOAD = "elast_64"
# It_max of the timed solves per workload (swept on GB300; see the design notes): (mixed, FP64)
# It_max of the timed path (and of the FP64 "compare" record).  64x64x32 box, mixed, GB300,
# one solve each: It_max 21 / 22 / 23 / 24 / 25 / 30 / 40 -> 28.5 / 29.1 / 29.5 / 28.4 / 28.9 /
# 23.5 / 18.2 eigenpairs/s (15 / 14 / 13 / 13 / 12 / 12 / 13 outer steps)
DEFAULT_IT_MAX = {"q1_lap_41": 8, "elast_32": 20, "elast_48": 20, "elast_64": 23, "bar1d_2000": 200}
DEFAULT_IT_MAX_FP64 = {"q1_lap_41": 8, "elast_32": 40, "elast_48": 40, "elast_64": 23, "bar1d_2000": 200}
# Jacobi preconditioner (D = diag(A), applied on both sides) on by default for the elasticity boxes
DEFAULT_PRECOND = {"elast_32": 1, "elast_48": 1, "elast_64": 1}
# DRAM bytes (read + write) of one full-width launch of the timed path's SpMM kernel, from
# an ncu capture of the kernel as it is now (block 32, 2 tiles, scaled to the 30 tiles of
# block 480; traffic is linear in the tiles), keyed by (workload, precision); an entry is
# dropped when the kernel changes.  The grouped kernel with B-diagonal records read 74.2 GB
# per launch when it staged 63-record chunks; the 81-record chunks it stages now have not
# been captured, so the roofline's traffic is null.
DEFAULT_TRAFFIC = {}


def measured_hbm_gbs():
    """Measured GB300 copy bandwidth (MEASURED_PEAKS.json at the repository root), else the
    fallback figure of an earlier measurement."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return float(json.load(fh)["hbm_gbs"]), "of measured"
    except Exception:
        return 6800.0, "of fallback"


def reduce_over_ranks(found: int, ms: float, world: int, device: str = "cuda"):
    """Whole-job totals of N independent replicas (one per GPU): eigenpairs summed over the
    ranks, time = the slowest rank's.  world == 1 returns the inputs."""
    if world <= 1:
        return found, ms
    import torch
    import torch.distributed as dist

    f = torch.tensor([float(found)], dtype=torch.float64, device=device)
    m = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(f, op=dist.ReduceOp.SUM)
    dist.all_reduce(m, op=dist.ReduceOp.MAX)
    return int(round(f.item())), float(m.item())


def workload(name: str, it_max: int | None):
    import slrf_inputs as si

    if name == "q1_lap_41":
        wl = si.q1_lap(41)
        wl.it_max = it_max or 8
        desc = ("3D Q1 Laplacian + consistent mass, 41^3 nodes (n=68,921, 27 nnz/row), Neumann + 1e-3 B, "
                "gamma=259.0666 (105 eigenpairs), block 160, m=8")
    elif name.startswith("q1_lap_"):
        nodes = int(name.split("_")[-1])
        wl = si.q1_lap(nodes)
        wl.it_max = it_max or 40
        desc = (f"3D Q1 Laplacian + consistent mass, {nodes}^3 nodes (n={wl.n}), Neumann + 1e-3 B, "
                f"gamma={wl.gamma:.4f} ({wl.n_expected} eigenpairs), block {wl.block}, m=8")
    elif name in ("elast_32", "elast_48", "elast_64"):
        from slrf_inputs import elastic as se

        p = se.pencil(name)
        g, cnt = se.gamma(name)
        spec = se.SPECS[name]
        wl = si.Workload(name, p, g, spec["block"], 8, spec["seed"], it_max or DEFAULT_IT_MAX.get(name, 40), cnt)
        nx, ny, nz = spec["nodes"]
        desc = (f"3D Q1 elasticity {nx}x{ny}x{nz} nodes, z=0 clamped (n={p.n:,}, nnz={p.nnz:,}, 3 dof/node), "
                f"E lognormal(0,0.5) seed {spec['seed']}, nu=0.3, rho=1, gamma={g:.6g} ({cnt} eigenpairs), "
                f"block {spec['block']}, m=8")
    elif name == "bar1d_2000":
        wl = si.bar1d(2000)
        wl.it_max = it_max or 200
        desc = "1D linear-FEM bar n=2000, gamma=4150.528 (20 eigenpairs), block 32, m=8"
    else:
        raise SystemExit(f"unknown workload {name}")
    return wl, desc


def clocks_start(raw_path: str | None = None):
    """Sample nvidia-smi clocks and throttle reasons every 200 ms until clocks_stop();
    the raw samples also go to raw_path when one is given."""
    try:
        f = open(raw_path or os.devnull, "w")
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                             stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        return p, f
    except Exception:
        return None, None


def clocks_stop(p, f, dev_index: int):
    if p is None:
        return None
    p.terminate()
    try:
        out, _ = p.communicate(timeout=5)
    except Exception:
        p.kill()
        out = ""
    sm, mx, reasons = [], [], set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.splitlines():
        parts = [x.strip() for x in line.split(",")]
        if len(parts) < 9 or parts[0] != str(dev_index):
            continue
        try:
            sm.append(float(parts[1]))
            mx.append(float(parts[2]))
        except ValueError:
            continue
        for nm, v in zip(names, parts[5:9]):
            if v.lower().startswith("active"):
                reasons.add(nm)
    if f is not None:
        f.write(out)
        f.close()
    if not sm:
        return None
    return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons), "samples": len(sm)}


_W = {}  # per-process state of the oracle workers


def _oracle_worker_init(path):
    """Process-pool initialiser: one BLAS thread per process, the pencil and the sampled
    start columns from the shared file (the workers are started with spawn)."""
    import numpy as np
    import scipy.sparse as sp

    d = np.load(path)
    n = int(d["n"])
    _W["A"] = sp.csr_matrix((d["valA"], d["col"], d["rowptr"]), shape=(n, n))
    _W["B"] = sp.csr_matrix((d["valB"], d["col"], d["rowptr"]), shape=(n, n))
    _W["V"] = d["V"]
    _W["theta"] = d["theta"]
    _W["gamma"] = float(d["gamma"])
    _W["m"] = int(d["m"])
    _W["precond"] = int(d["precond"])


def _oracle_worker_filter(task):
    """The oracle's filter apply (all m poles, `its` COCG updates, warm start) on columns
    [lo, hi) of the sample; returns the COCG updates it performed."""
    lo, hi, its = task
    from oracle import slrf_oracle as orc

    A, B = _W["A"], _W["B"]
    sig, w = orc.slrf_poles(_W["m"], _W["gamma"])
    d = A.diagonal() if _W["precond"] else None
    _, info = orc.filter_apply(A, B, _W["V"][:, lo:hi], _W["theta"][lo:hi], sig, w, its, 1e-10, d)
    return int(info.iters.sum())


def cpu_baseline_sample(name: str, it_max: int, precond: int, n_found: int, col_iters: int, outer: int,
                        col_solves: int, m: int = 8, budget_s: float = 25.0):
    """The FP64 oracle, as it stands, on a bounded sample of the workload, on every host core,
    scaled to one whole solve with the counts of the GPU solve of the same run.

    Sample: (i) the oracle's warm-started filter apply (Alg. 2; theta spread over (0, gamma])
    on one start-block column per core, all m poles, a few COCG updates each, the columns in
    a spawn-started process pool of os.cpu_count() processes with one BLAS thread each ->
    seconds per column-iteration with every core busy; (ii) one Cholesky-QR2 + Rayleigh-Ritz
    step of the oracle on a column subset with all cores in BLAS, its sparse part scaled
    linearly and its dense part quadratically to the solve's mean active block.  Estimate:
    column-iterations x (i) + outer iterations x (ii)."""
    import multiprocessing as mp
    import tempfile

    import numpy as np

    import slrf_inputs as si
    from oracle import slrf_oracle as orc

    cores = os.cpu_count() or 1
    wl, _ = workload(name, it_max)
    p = wl.pencil
    k = wl.block
    V1 = si.start_block(p.n, k, wl.seed)
    c = min(k, cores)
    cols = np.ascontiguousarray(V1[:, :c])
    theta = (np.arange(c) + 0.5) / c * wl.gamma
    tmp = tempfile.NamedTemporaryFile(suffix=".npz", delete=False)
    tmp.close()
    np.savez(tmp.name, n=p.n, rowptr=p.rowptr, col=p.col, valA=p.valA, valB=p.valB, V=cols, theta=theta,
             gamma=wl.gamma, m=m, precond=precond)
    env_keep = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")}
    for v in env_keep:
        os.environ[v] = "1"
    try:
        ctx = mp.get_context("spawn")
        with ctx.Pool(processes=c, initializer=_oracle_worker_init, initargs=(tmp.name,)) as pool:
            pool.map(_oracle_worker_filter, [(j, j + 1, 1) for j in range(c)])  # load, warm up
            its_sample = 1
            t0 = time.perf_counter()
            its = sum(pool.map(_oracle_worker_filter, [(j, j + 1, its_sample) for j in range(c)]))
            t1 = time.perf_counter() - t0
            its_sample = int(max(1, min(it_max, (budget_s * 0.6) / max(t1, 1e-3))))
            t0 = time.perf_counter()
            its = sum(pool.map(_oracle_worker_filter, [(j, j + 1, its_sample) for j in range(c)]))
            t_f = time.perf_counter() - t0
    finally:
        for v, old in env_keep.items():
            if old is None:
                os.environ.pop(v, None)
            else:
                os.environ[v] = old
        os.unlink(tmp.name)
    per_it = t_f / max(its, 1)
    # (ii) one outer update on c_rr columns (all cores in BLAS), sparse and dense parts apart
    A, B = p.A(), p.B()
    c_rr = min(k, 96)
    U = np.ascontiguousarray(V1[:, :c_rr])
    t0 = time.perf_counter()
    A @ U
    B @ U
    B @ U
    t_sp = time.perf_counter() - t0
    t0 = time.perf_counter()
    Q, _ = orc.cholqr2(U, B)
    orc.rayleigh_ritz(Q, A)
    t_rr = time.perf_counter() - t0
    k_mean = max(1.0, col_solves / max(m * outer, 1))
    t_step = t_sp * (k_mean / c_rr) + max(t_rr - t_sp, 0.0) * (k_mean / c_rr) ** 2
    est = col_iters * per_it + outer * t_step
    return {"value": n_found / est, "unit": "eigenpairs/s", "cores": cores, "kind": "oracle",
            "sample": (f"oracle warm-started filter apply of {c} of {k} start columns x {m} poles x {its_sample} COCG "
                       f"updates ({its} column-iterations in {t_f:.1f} s, one column per process, {c} processes on "
                       f"{cores} cores) + one Cholesky-QR2/Rayleigh-Ritz step on {c_rr} columns ({t_rr:.1f} s, "
                       f"BLAS on all cores), scaled to this run's GPU solve: {col_iters} column-iterations and "
                       f"{outer} outer iterations at a mean active block of {k_mean:.0f}"),
            "seconds_sampled": t_f + t_rr + t_sp}


def spmm_roofline(p, m: int, k: int, precision: int, spmm_ms: float, traffic, bdiag: bool = False):
    """Roofline of the fused shifted SpMM + COCG phase-1 launch (the dominant kernel) at k
    columns x m poles: algorithmic flops 8 per (entry of the shared pattern, complex column)
    + 32 per (row, complex column), algorithmic bytes 5 complex entries per (row, column) (r,
    p, q read; p, q written) + one pass over the pattern and both value arrays.  With
    B-diagonal records the kernel multiplies only B's nonzero entries, so its executed flops
    count 4 per pattern entry (A) + 4 per nonzero of B; the ALU side of the roofline uses the
    executed flops.  The bound is whichever of the ALU (FP64 / FP32 FMA pipe) and HBM times is
    larger."""
    W = m * k
    es = 16 if precision == 0 else 8
    flops_alg = 8.0 * p.nnz * W + 32.0 * p.n * W
    nnz_b = int((p.valB != 0).sum())
    flops = (4.0 * p.nnz + 4.0 * nnz_b) * W + 32.0 * p.n * W if bdiag else flops_alg
    nbytes = 5.0 * es * p.n * W + p.nnz * (4 + 2 * (8 if precision == 0 else 4))
    hbm, hbm_note = measured_hbm_gbs()
    alu_peak = FP64_PEAK_TFLOPS if precision == 0 else FP32_PEAK_TFLOPS
    t_alu = flops / (alu_peak * 1e12)
    t_hbm = nbytes / (hbm * 1e9)
    s = spmm_ms / 1e3
    kern = "cocg SpMM, FP64" if precision == 0 else "cocg SpMM, FP32 (grouped-row kernel when the format has groups)"
    if t_alu >= t_hbm:
        achieved = flops / s / 1e12
        return {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s", "frac": achieved / alu_peak,
                "traffic": traffic, "kernel": kern,
                "note": (f"FP{64 if precision == 0 else 32} FMA pipe bound ({flops / nbytes:.1f} flop/B); peak = 152 SMs "
                         f"x {2 if precision == 0 else 128} FMA/clock x 2 x 2.07 GHz (derived); HBM "
                         f"{nbytes / s / 1e9:.0f} GB/s = {nbytes / s / 1e9 / hbm:.2f} {hbm_note} {hbm:.0f} GB/s"),
                "hbm_gbs_algorithmic": nbytes / s / 1e9, "flops_per_launch": flops, "flops_pattern_per_launch": flops_alg,
                "bytes_per_launch": nbytes, "b_diagonal_records": bdiag}
    achieved = nbytes / s / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": traffic, "kernel": kern,
            "note": (f"{hbm_note} hbm_gbs; {flops / s / 1e12:.1f} TFLOP/s executed "
                     f"({flops / s / 1e12 / alu_peak:.2f} of the FP{64 if precision == 0 else 32} peak)"
                     + ("; B-diagonal records: only B's nonzeros multiplied" if bdiag else "")),
            "flops_per_launch": flops, "flops_pattern_per_launch": flops_alg, "bytes_per_launch": nbytes,
            "b_diagonal_records": bdiag}


def paper_table_records(slrf, si, torch):
    """Two small-problem records on the Q1 Laplacian with 21^3 nodes (n = 9,261, gamma
    enclosing about 100 eigenvalues, block 1.5x, m = 8, FP64), analogues of the paper's:
      * Table 3: enhanced Alg. 2 (locking, warm start, It_max 8) against the basic Alg. 1
        (no locking, zero initial guesses, inner solves to 1e-13 or 2000 updates) -- the
        time ratio of the two whole solves;
      * Table 1 "Ratio": per-pole spread of the COCG updates needed to reach 1e-10 from the
        zero guess (start block, up to 5000 updates) for the SLRF poles and for the
        midpoint / Gauss-Legendre / Gauss-Chebyshev contour filters (pole tables through
        slrf_opts.poles), max/min over poles of the mean updates, and each table's whole
        enhanced solve."""
    import numpy as np

    wl = si.q1_lap(21)
    p = wl.pencil
    V0 = torch.from_numpy(si.start_block(p.n, wl.block, wl.seed)).cuda()

    def solve(**kw):
        ctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, wl.gamma, wl.block, slrf.slrf_opts_default(**kw))
        ctx.solve(V0, check=False)  # warm-up (graph capture, module loading)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        rc, nf, ev, X, rs, st = ctx.solve(V0, check=False)
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        ctx.close()
        return {"rc": rc, "eigenpairs": nf, "outer_iters": st["outer_iters"], "seconds": dt,
                "column_iterations": st["column_iterations"],
                "max_resid": float(rs.max().item()) if nf else None}

    enh = solve(it_max=8)
    basic = solve(it_max=2000, tol_inner=1e-13, lock=0, warm_start=0, outer_max=60)
    t3 = {"workload": f"q1_lap_21: 3D Q1 Laplacian 21^3 nodes (n={p.n}), gamma={wl.gamma:.4f} "
                      f"({wl.n_expected} eigenpairs), block {wl.block}, m=8, FP64",
          "enhanced_alg2": enh, "basic_alg1": basic,
          "time_ratio_basic_over_enhanced": basic["seconds"] / enh["seconds"]}
    t1 = {}
    for rule in ("slrf", "midpoint", "gauss_legendre", "gauss_chebyshev"):
        kw = {}
        if rule != "slrf":
            s_, w_ = slrf.quadrature_table(rule, 8, wl.gamma)
            kw = {"poles": s_, "weights": w_}
        ctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, wl.gamma, wl.block,
                           slrf.slrf_opts_default(it_max=5000, **kw))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ctx.filter_apply(V0)
        torch.cuda.synchronize()
        tf = time.perf_counter() - t0
        its, rr, bk = ctx.filter_stats(wl.block)
        ctx.close()
        per_pole = its.mean(axis=1)
        rec = {"per_pole_mean_updates": [float(x) for x in per_pole],
               "ratio_max_over_min": float(per_pole.max() / per_pole.min()),
               "converged_columns": int(np.sum(rr <= 1e-10)), "filter_seconds": tf,
               "enhanced_solve": solve(it_max=8, **kw)}
        t1[rule] = rec
    return {"alg1_vs_alg2": t3, "pole_tables": t1}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=DEFAULT_WORKLOAD)
    ap.add_argument("--it-max", type=int, default=None, help="It_max of the timed path (default per workload)")
    ap.add_argument("--precision", type=int, default=1,
                    help="timed path: 1 = complex-FP32 COCG in FP64 refinement (default), 0 = FP64 throughout")
    ap.add_argument("--precond", type=int, default=None, help="Jacobi-preconditioned inner solves (default per workload)")
    ap.add_argument("--group", type=int, default=0, help="rows per group of the COCG SpMM (0 = chosen at setup)")
    ap.add_argument("--compare-steps", type=int, default=1,
                    help="timed solves of the other precision on the same workload (0 = skip)")
    ap.add_argument("--compare-it-max", type=int, default=None)
    ap.add_argument("--e2e-steps", type=int, default=2, help="whole solves from host buffers for the e2e figure")
    ap.add_argument("--traffic-bytes", type=float, default=None,
                    help="DRAM bytes of one SpMM launch from an ncu capture of the current kernel (else null)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--filter-only", type=int, default=0, metavar="L",
                    help="profiling aid: kernel-by-kernel timing of filter applies with block L, no JSON line")
    ap.add_argument("--solve-once", action="store_true",
                    help="profiling aid: one solve at the bench settings (for launch lists), no JSON line")
    ap.add_argument("--counts-out", default=None,
                    help="write the timed solve's counts (the reference arm's scaling) to this JSON file")
    ap.add_argument("--no-tables", action="store_true",
                    help="skip the small-problem records of the paper's Tables 1 and 3")
    ap.add_argument("--clocks-csv", default=None,
                    help="also write the raw nvidia-smi clock samples of the timed region to this file")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="batch64: also time the plain FP64 batched solve")
    ap.add_argument("--mixed-it-max", type=int, default=8, help="batch64 / sens48: It_max of the mixed path")
    ap.add_argument("--dense", type=int, default=1,
                    help="1: FP64-accurate split-bf16 tensor-core products in the outer update; 0: FP64 FMA")
    ap.add_argument("--it-adapt", type=int, default=0,
                    help="1: per-problem It_max grows while the lowest active Ritz pair is unresolved")
    ap.add_argument("--directions", type=int, default=8,
                    help="sens48: random directions of the finite-difference check")
    args = ap.parse_args()

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        return reference_arm(args, rank, world)
    if args.workload == "batch64":
        return batch_bench(args, rank, world, local)
    if args.workload == "sens48":
        return sens_bench(args, rank, world, local)

    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__ as ge

    ge.build()
    import slrf_inputs as si
    from paper_2510_17334_gb300 import slrf

    prec = args.precision
    it_main = args.it_max or (DEFAULT_IT_MAX if prec == 1 else DEFAULT_IT_MAX_FP64).get(args.workload, 40)
    wl, desc = workload(args.workload, it_main)
    p = wl.pencil
    precond = DEFAULT_PRECOND.get(args.workload, 0) if args.precond is None else args.precond
    stream = torch.cuda.Stream()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def timed_solves(precision, it_max, steps, warmup, clocks=False):
        opts = slrf.slrf_opts_default(m=wl.m, it_max=it_max, precision=precision, dense=args.dense, precond=precond,
                                      group=args.group)
        with torch.cuda.stream(stream):
            ctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, wl.gamma, wl.block, opts, stream=stream)
            V0 = torch.from_numpy(si.start_block(p.n, wl.block, wl.seed)).cuda()
            for _ in range(warmup):
                ctx.solve(V0)
            barrier()
            cp, cf = clocks_start(args.clocks_csv) if clocks else (None, None)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            found, stats, last = [], [], None
            e0.record(stream)
            for _ in range(steps):
                last = ctx.solve(V0)
                found.append(last[1])
                stats.append(last[5])
            e1.record(stream)
            barrier()
            clk = clocks_stop(cp, cf, local) if clocks else None
            ms = e0.elapsed_time(e1)
        return ctx, V0, found, stats, last, ms, clk

    if args.filter_only or args.solve_once:
        return profile_aid(args, slrf, si, wl, prec, it_main, precond, stream)

    # ---- the timed path
    ctx, V0, found, stats, last, ms, clk = timed_solves(prec, it_main, args.steps, args.warmup, clocks=True)
    total_found, ms_max = reduce_over_ranks(sum(found), ms, world)
    rc, nf, ev, X, rs, st = last
    maxres = float(rs.max().item())
    # kernel-level roofline of the dominant kernel (the fused shifted SpMM + COCG phase 1)
    with torch.cuda.stream(stream):
        tim = ctx.filter_timing(V0[:, :wl.block])
    fmt = ctx.format()
    ctx.close()
    spmm_ms = tim["ms_spmm"] / max(tim["n_spmm"], 1)
    traffic = args.traffic_bytes
    if traffic is None and args.group == 0:
        traffic = DEFAULT_TRAFFIC.get((args.workload, prec))
    roof = spmm_roofline(p, wl.m, wl.block, prec, spmm_ms, traffic, bdiag=fmt[1] == 1)
    roof["spmm_format"] = {"group": fmt[0], "b_diagonal": fmt[1], "lane_width": fmt[2]}
    roof["update_ms"] = tim["ms_update"] / max(tim["n_update"], 1)
    roof["spmm_ms"] = spmm_ms
    # ---- the other precision on the same workload (FP64 vs mixed at equal residual)
    compare = None
    if args.compare_steps > 0:
        cprec = 1 - prec
        cit = args.compare_it_max or (DEFAULT_IT_MAX if cprec == 1 else DEFAULT_IT_MAX_FP64).get(args.workload, 40)
        cctx, _, cfound, cstats, clast, cms, _ = timed_solves(cprec, cit, args.compare_steps, 0)
        cctx.close()
        ctot, cms = reduce_over_ranks(sum(cfound), cms, world)
        cev = clast[2].cpu().numpy()
        fev = ev.cpu().numpy()
        diff = float(np.max(np.abs(cev - fev) / np.abs(fev))) if len(cev) == len(fev) and len(fev) else None
        compare = {"precision": cprec, "value": ctot / (cms / 1e3), "unit": "eigenpairs/s", "it_max": cit,
                   "steps": args.compare_steps, "warmup": 0, "ms_per_step": cms / args.compare_steps,
                   "eigenpairs_found": clast[1], "max_resid": float(clast[4].max().item()) if clast[1] else None,
                   "max_rel_eig_diff": diff, "outer_iters": clast[5]["outer_iters"],
                   "ms_filter_per_step": clast[5]["ms_filter"], "ms_dense_per_step": clast[5]["ms_dense"]}
    # ---- end to end through the host-buffer entry point (setup + solve + copies per step)
    opts = slrf.slrf_opts_default(m=wl.m, it_max=it_main, precision=prec, dense=args.dense, precond=precond,
                                  group=args.group)
    pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
    hrp, hcol, hA, hB = pin(p.rowptr), pin(p.col.astype(np.int32)), pin(p.valA), pin(p.valB)
    hV0 = pin(si.start_block(p.n, wl.block, wl.seed))
    e2e_found, e2e_s = 0, 0.0
    torch.cuda.synchronize()
    for _ in range(max(1, args.e2e_steps)):
        t0 = time.perf_counter()
        ev_h, X_h, rs_h, st_h = slrf.slrf_solve_host(hrp, hcol, hA, hB, wl.gamma, wl.block, opts, hV0)
        e2e_s += time.perf_counter() - t0
        e2e_found += len(ev_h)
    h2d = hrp.nbytes + hcol.nbytes + hA.nbytes + hB.nbytes + hV0.nbytes
    d2h = 2 * 8 * wl.block + p.n * wl.block * 8
    value = total_found / (ms_max / 1e3)
    col_solves = sum(s["column_solves"] for s in stats)
    col_iters = sum(s["column_iterations"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    W = wl.m * wl.block
    es = 16 if prec == 0 else 8
    line = {
        "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if prec == 0 else "c32 inner solves in f64 refinement",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "it_max": it_main, "precision": prec, "precond": precond,
                   "group": args.group,
                   "l2": "inputs larger than L2 (COCG state %.1f GB)" % (4 * es * p.n * W / 1e9),
                   "parallelism": f"replicas x{world}"},
        "column_solves_per_s": col_solves * world / (ms_max / 1e3),
        "column_iterations_per_s": col_iters * world / (ms_max / 1e3),
        "spmm_gbs_algorithmic": roof.get("hbm_gbs_algorithmic", roof["achieved"]),
        "eigenpairs_found": nf, "eigenpairs_expected": wl.n_expected, "max_resid": maxres, "rc": rc,
        "outer_iters": st["outer_iters"],
        "ms_filter_per_step": sum(s["ms_filter"] for s in stats) / args.steps,
        "ms_dense_per_step": sum(s["ms_dense"] for s in stats) / args.steps,
        "roofline": roof,
        "e2e": {"value": e2e_found / e2e_s, "unit": "eigenpairs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h), "steps": max(1, args.e2e_steps)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "compare": compare,
    }
    if rank == 0 and world == 1 and not args.no_tables:
        line["paper_tables"] = paper_table_records(slrf, si, torch)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(args.workload, it_main, precond, nf,
                                                       int(col_iters / args.steps), st["outer_iters"],
                                                       int(col_solves / args.steps), wl.m)
    if rank == 0 and args.counts_out:
        rec = {"it_max": it_main, "precond": precond, "precision": prec, "n_found": nf,
               "column_iterations": int(col_iters / args.steps), "outer": st["outer_iters"],
               "column_solves": int(col_solves / args.steps)}
        with open(args.counts_out, "w") as fh:
            json.dump({args.workload: rec}, fh, indent=1)
    if rank == 0:
        print(json.dumps(line))
    if world > 1:
        torch.distributed.destroy_process_group()


def profile_aid(args, slrf, si, wl, prec, it_main, precond, stream):
    """Small, self-contained runs to profile under ncu (no JSON line): --filter-only L times
    3 filter applies of the workload with block L (It_max 4, launch by launch, CUDA events);
    --solve-once runs one solve at the bench settings."""
    import torch

    p = wl.pencil
    L = args.filter_only or wl.block
    opts = slrf.slrf_opts_default(m=wl.m, it_max=4 if args.filter_only else it_main, precision=prec,
                                  dense=args.dense, precond=precond, group=args.group)
    with torch.cuda.stream(stream):
        ctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, wl.gamma, L, opts, stream=stream)
        V0 = torch.from_numpy(si.start_block(p.n, L, wl.seed)).cuda()
        if args.filter_only:
            for _ in range(3):
                tm = ctx.filter_timing(V0)
            print(f"{args.workload} block {L} precision {prec}: SpMM {tm['ms_spmm'] / max(tm['n_spmm'], 1):.3f} ms, "
                  f"update {tm['ms_update'] / max(tm['n_update'], 1):.3f} ms, filter {tm['ms_total']:.2f} ms")
        else:
            t0 = time.perf_counter()
            rc, nf, ev, X, rs, st = ctx.solve(V0)
            torch.cuda.synchronize()
            print(f"{args.workload} precision {prec}: rc {rc}, {nf} eigenpairs, {time.perf_counter() - t0:.2f} s, "
                  f"{st['outer_iters']} outer iterations, {st['kernel_launches']} launches")
        ctx.close()


def batch_bench(args, rank, world, local):
    """64 uneven scalar Q1 pencils (slrf_inputs.batch) solved together: the COCG phases of
    all problems in one persistent launch per phase.  A step = one batched solve."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    import __graft_entry__ as ge

    ge.build()
    import slrf_inputs as si
    from slrf_inputs import batch as sb
    from paper_2510_17334_gb300 import slrf

    specs = sb.batch_specs()
    gam = sb.batch_gammas()
    pens = [sb.batch_pencil(s) for s in specs]
    probs = [(p.rowptr, p.col, p.valA, p.valB) for p in pens]
    gammas = [g for g, _ in gam]
    counts = [c for _, c in gam]
    blocks = [int(np.ceil(1.5 * c)) for c in counts]
    V0 = [torch.from_numpy(si.start_block(p.n, L, s.seed)).cuda() for p, L, s in zip(pens, blocks, specs)]
    stream = torch.cuda.Stream()

    def run(precision, it_max):
        opts = slrf.slrf_opts_default(it_max=it_max, precision=precision, autotune=1, it_adapt=args.it_adapt,
                                      dense=args.dense)
        with torch.cuda.stream(stream):
            b = slrf.Batch(probs, gammas, blocks, opts, stream=stream)
            for _ in range(args.warmup):
                b.solve(V0, check=False)
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            found = 0
            for _ in range(args.steps):
                rc, res, st = b.solve(V0, check=False)
                found += sum(r[1] for r in res)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1)
            exact = sum(1 for r, c in zip(res, counts) if r[1] == c)
            maxres = max(float(r[4].max().item()) for r in res if r[1] > 0)
            evs = [r[2].cpu().numpy() for r in res]
            b.close()
        return {"value": found / (ms / 1e3), "ms_per_step": ms / args.steps, "rc": rc,
                "problems_with_exact_count": exact, "eigenpairs": found // args.steps, "max_resid": maxres,
                "outer_iters_max": st["outer_iters"], "column_iterations": st["column_iterations"],
                "ms_cocg_per_step": st["ms_filter"], "ms_rest_per_step": st["ms_dense"],
                "kernel_launches": st["kernel_launches"], "it_max": it_max}, evs

    cp, cf = clocks_start(args.clocks_csv)
    prec = 1 if args.precision == 0 and not args.compare_fp64 else args.precision
    main, evs_main = run(1, args.mixed_it_max if args.it_max is None else args.it_max)
    clk = clocks_stop(cp, cf, local)
    fp64 = None
    if args.compare_fp64:
        fp64, evs64 = run(0, args.it_max or args.mixed_it_max)
        diffs = [float(np.max(np.abs(a - b) / np.abs(b))) for a, b in zip(evs_main, evs64) if len(a) == len(b) and len(a)]
        fp64["max_rel_eig_diff_mixed_vs_fp64"] = max(diffs) if diffs else None
    ntot = sum(p.n for p in pens)
    line = {"metric": METRIC, "value": main["value"], "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": main["ms_per_step"], "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "c32-in-f64", "data": "synthetic",
            "config": {"workload": (f"batch64: 64 uneven scalar Q1 pencils (2D/3D, lognormal(0,0.3) coefficients, "
                                    f"sum n = {ntot}, {sum(counts)} eigenpairs, blocks 1.5x count, m=8), "
                                    f"one persistent COCG launch per phase"),
                       "precision": "mixed (complex-FP32 COCG, FP64 outer)", "autotune": 1,
                       "it_adapt": args.it_adapt},
            "batched_mixed": main, "batched_fp64": fp64, "gpu_launches": main["kernel_launches"], "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


def sens_bench(args, rank, world, local):
    """Eigenvalue sensitivity of the 48^3 Q1 elasticity box: lowest 50 eigenpairs (mixed
    path), loss L = sum_i c_i lambda_i, c ~ N(0, 1), and its gradient with respect to the
    per-element stiffness parameters p_e through the eigenvalue adjoint (slrf_eig_grad).
    A = sum_e p_e K_e is linear in p, so for a direction dp the directional derivative is
    <gA, values of A assembled with p = dp> (B does not depend on p).  It is checked against
    the closed form sum_i c_i x_i^T dA x_i and against central differences of L at
    p +- h dp (h = 1e-6, relative directions dp = p .* N(0, 1)), each a warm-started solve."""
    import numpy as np
    import torch

    torch.cuda.set_device(local)
    import __graft_entry__ as ge

    ge.build()
    from slrf_inputs import elastic as se
    from paper_2510_17334_gb300 import slrf

    name = "elast_48"
    spec = se.SPECS[name]
    pe = se.element_params(name)
    P0 = se.pencil(name, pe)
    gamma, cnt = se.gamma(name)
    L = spec["block"]
    rng = np.random.default_rng(11)
    cvec = rng.standard_normal(cnt)
    it = args.it_max or 20
    opts = slrf.slrf_opts_default(it_max=it, precision=1, tol_eig=1e-9)
    V0 = torch.from_numpy(__import__("slrf_inputs").start_block(P0.n, L, spec["seed"])).cuda()

    def solve(valA, V):
        ctx = slrf.Context(P0.rowptr, P0.col, valA, P0.valB, gamma, L, opts)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        rc, nf, ev, X, rs, st = ctx.solve(V, check=False)
        e1.record()
        torch.cuda.synchronize()
        return ctx, rc, nf, ev, X, rs, st, e0.elapsed_time(e1)

    cp, cf = clocks_start(args.clocks_csv)
    ctx, rc, nf, ev, X, rs, st, ms_solve = solve(P0.valA, V0)
    assert rc == 0 and nf == cnt, (rc, nf, cnt)
    cd = torch.from_numpy(cvec).cuda()
    ctx.eig_grad(ev, X, cd)  # warm-up
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    gA, gB = ctx.eig_grad(ev, X, cd)
    e1.record()
    torch.cuda.synchronize()
    ms_adj = e0.elapsed_time(e1)
    ctx.close()
    Xh = X.cpu().numpy()
    evh = ev.cpu().numpy()
    gAh = gA.cpu().numpy()
    L0 = float(cvec @ evh)
    # warm start of the perturbed solves: the eigenvectors plus Gaussian columns
    Vw = V0.clone()
    Vw[:, :cnt] = X
    A0 = P0.A().tocsr()
    h = 1e-6
    err_cf, err_fd, rows = [], [], []
    for d in range(args.directions):
        dp = pe * rng.standard_normal(pe.size)
        dP = se.pencil(name, dp)
        assert np.array_equal(dP.rowptr, P0.rowptr) and np.array_equal(dP.col, P0.col)
        g_adj = float(gAh @ dP.valA)
        dA = dP.A().tocsr()
        g_cf = float(np.sum(cvec * np.einsum("ij,ij->j", Xh, dA @ Xh)))
        Ls = []
        for sgn in (1.0, -1.0):
            c2, rc2, nf2, ev2, X2, rs2, st2, _ = solve(P0.valA + sgn * h * dP.valA, Vw)
            c2.close()
            assert rc2 == 0 and nf2 == cnt, (rc2, nf2)
            Ls.append(float(cvec @ ev2.cpu().numpy()))
        g_fd = (Ls[0] - Ls[1]) / (2 * h)
        err_cf.append(abs(g_adj - g_cf) / abs(g_cf))
        err_fd.append(abs(g_adj - g_fd) / abs(g_fd))
        rows.append({"adjoint": g_adj, "closed_form": g_cf, "central_fd": g_fd})
    clk = clocks_stop(cp, cf, local)
    line = {"metric": "eigenvalue-sensitivity gradient dL/dp vs closed form and central differences",
            "value": max(err_fd) if err_fd else None, "unit": "max relative error (central FD)",
            "n_gpus": 1, "higher_is_better": False, "data": "synthetic", "dtype": "f64 (adjoint), c32-in-f64 (solve)",
            "config": {"workload": (f"sens48: 3D Q1 elasticity 48^3 nodes, z=0 clamped (n={P0.n}, nnz={P0.nnz}), "
                                    f"p_e lognormal(0,0.5) seed {spec['seed']}, lowest {cnt} eigenpairs, block {L}, "
                                    f"L = sum c_i lambda_i, c ~ N(0,1) seed 11"),
                       "it_max": it, "h": h, "directions": args.directions},
            "solve": {"ms": ms_solve, "eigenpairs": nf, "max_resid": float(rs.max().item()),
                      "outer_iters": st["outer_iters"], "loss": L0},
            "adjoint": {"ms": ms_adj, "nnz": P0.nnz, "eigenpairs": cnt,
                        "gbs_algorithmic": (P0.nnz * (8 + 8 + 12) + P0.n * cnt * 8) / (ms_adj * 1e6)},
            "max_rel_err_vs_closed_form": max(err_cf) if err_cf else None,
            "max_rel_err_vs_central_fd": max(err_fd) if err_fd else None,
            "directions_detail": rows, "clocks": clk}
    if rank == 0:
        print(json.dumps(line))


def cpu_baseline_subprocess(name, it_max, precond, n_found, col_iters, outer, col_solves, m):
    """cpu_baseline_sample in a fresh process (its pool starts with spawn; no CUDA there)."""
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline_sample(%r, %d, %d, %d, %d, %d, %d, %d)))" %
            (ROOT, name, it_max, precond, n_found, col_iters, outer, col_solves, m))
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=900)
    try:
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return {"value": None, "error": r.stderr[-300:]}


def solve_counts(name: str):
    """Counts of one solve of the workload by Alg. 2 at the timed settings (outer iterations,
    column-iterations, column-solves, eigenpairs), stored with the workload inputs
    (slrf_inputs/solve_counts.json); the oracle performs the same counts (the parity tests
    check identical COCG update counts), so they scale the oracle's timed sample."""
    path = os.path.join(ROOT, "slrf_inputs", "solve_counts.json")
    try:
        with open(path) as fh:
            return json.load(fh).get(name)
    except Exception:
        return None


def reference_arm(args, rank, world):
    """The oracle as it stands on the host cores, same workload, metric and unit.  Each step
    is a bounded sample (cpu_baseline_sample: every core busy) scaled to one whole solve
    with the workload's solve counts.  Under torchrun only rank 0 works."""
    if rank != 0:
        return
    cnt = solve_counts(args.workload)
    if cnt is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no solve counts recorded for {args.workload}"}))
        return
    wl, desc = workload(args.workload, cnt["it_max"])
    vals = []
    t_start = time.perf_counter()
    for s in range(args.warmup + args.steps):
        r = cpu_baseline_sample(args.workload, cnt["it_max"], cnt.get("precond", 0), cnt["n_found"],
                                cnt["column_iterations"], cnt["outer"], cnt["column_solves"], wl.m, budget_s=6.0)
        if s >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    line = {"metric": METRIC, "value": v, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": (time.perf_counter() - t_start) * 1e3 / (args.warmup + args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "it_max": cnt["it_max"],
                       "precision": 0, "precond": cnt.get("precond", 0),
                       "counts_from": ("the GPU solve at these settings, precision %d (outer iterations, "
                                       "column-iterations, mean active block)" % cnt.get("precision", 0)),
                       "l2": "n/a (host)", "parallelism": "replicas x1"},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "eigenpairs/s", "cores": vals[-1]["cores"], "kind": "oracle",
                             "sample": vals[-1]["sample"].replace("this run's GPU solve", "the recorded solve")},
            "e2e": {"value": v, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
