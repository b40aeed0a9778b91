"""Benchmark of the SLRF hot path (enhanced ParaSLRF, Alg. 2) on one GB300.

One step = one slrf_solve of the workload: every outer iteration's filter apply (all
poles x columns by COCG), B-orthogonalisation against the locked vectors, Cholesky-QR2,
Rayleigh-Ritz, residuals, locking and the warm start.  Default workload: the 3D Q1
Laplacian on 41^3 nodes (n = 68,921, 27 nnz/row), gamma = 259.0666 (105 eigenpairs),
block 160, m = 8 poles, FP64.

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

METRIC = "eigenpairs/s and shifted column-solves/s at resid≤1e-8; SpMM HBM GB/s vs peak"
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12  # 152 SMs x 2 FP64 FMA/clock x 2 flops x 2.07 GHz
# DRAM bytes (read + write) of one cocg_spmm_kernel<double> launch on the 41^3 workload at
# 160 columns x 8 poles, from the ncu capture summarised in profiles/launches_q1_lap_41_fp64.md
SPMM64_TRAFFIC_Q1_41 = 5978269696 + 2815613952


# Counts of one solve of each workload by Alg. 2 (column-iterations = COCG updates summed
# over all (pole, column) systems and outer iterations), used to scale the timed oracle
# sample of the reference arm to a whole solve.
SOLVE_COUNTS = {"q1_lap_41": {"n_found": 105, "outer": 18, "column_iterations": 145920},
                "bar1d_2000": {"n_found": 20, "outer": 8, "column_iterations": 358400},
                "elast_32": {"n_found": 60, "outer": 20, "column_iterations": 448640}}


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
    elif name in ("elast_32", "elast_48"):
        from slrf_inputs import elastic as se

        p = se.pencil(name)
        g, cnt = se.gamma(name)
        spec = se.SPECS[name]
        wl = si.Workload(name, p, g, spec["block"], 8, spec["seed"], it_max or 40, cnt)
        desc = (f"3D Q1 elasticity {spec['nodes']} nodes, z=0 clamped (n={p.n}, nnz={p.nnz}), E lognormal(0,0.5), "
                f"nu=0.3, gamma={g:.4f} ({cnt} eigenpairs), block {spec['block']}, m=8")
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


def cpu_baseline_sample(name: str, it_max: int, n_found: int, col_iters: int, outer: int, budget_s: float = 20.0):
    """Time the oracle on a bounded sample of the workload and scale it to eigenpairs/s.

    Sample: the oracle's filter apply on the first c start-block columns (all m poles,
    It_max COCG updates) and one Rayleigh-Ritz step on the full block.  The estimate
    scales the per-column-iteration time by the column-iterations and the RR time by the
    outer iterations that the GPU solve of the same workload performed."""
    import numpy as np

    import slrf_inputs as si
    from oracle import slrf_oracle as orc

    wl, _ = workload(name, it_max)
    p = wl.pencil
    A, B = p.A(), p.B()
    V1 = si.start_block(p.n, wl.block, wl.seed)
    sig, w = orc.slrf_poles(wl.m, wl.gamma)
    c = 1
    t0 = time.perf_counter()
    _, info = orc.filter_apply(A, B, V1[:, :c], None, sig, w, wl.it_max, 1e-10)
    t_f = time.perf_counter() - t0
    # grow the sample while it stays within the budget
    if t_f < budget_s / 4:
        c = max(1, min(wl.block, int(c * (budget_s / 2) / max(t_f, 1e-3))))
        t0 = time.perf_counter()
        _, info = orc.filter_apply(A, B, V1[:, :c], None, sig, w, wl.it_max, 1e-10)
        t_f = time.perf_counter() - t0
    its = int(info.iters.sum())
    t0 = time.perf_counter()
    U, _ = orc.cholqr2(V1.copy(), B)
    orc.rayleigh_ritz(U, A)
    t_rr = time.perf_counter() - t0
    per_it = t_f / max(its, 1)
    est = col_iters * per_it + outer * t_rr
    return {"value": n_found / est, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
            "sample": (f"oracle filter apply of {c} of {wl.block} columns x {wl.m} poles x It_max={wl.it_max} "
                       f"({its} column-iterations, {t_f:.1f} s) + one CholQR2/RR step on the full block "
                       f"({t_rr:.1f} s), scaled to the GPU solve's {col_iters} column-iterations and "
                       f"{outer} outer iterations"),
            "seconds_sampled": t_f + t_rr}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="q1_lap_41")
    ap.add_argument("--it-max", type=int, default=None)
    ap.add_argument("--precision", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--clocks-csv", default=None,
                    help="also write the raw nvidia-smi clock samples of the timed region to this file")
    ap.add_argument("--compare-fp64", action="store_true",
                    help="batch64: also time the plain FP64 batched solve")
    ap.add_argument("--mixed-it-max", type=int, default=8,
                    help="It_max of the complex-FP32 inner solves for the mixed-path line (0 = skip)")
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

    wl, desc = workload(args.workload, args.it_max)
    p = wl.pencil
    opts = slrf.slrf_opts_default(m=wl.m, it_max=wl.it_max, precision=args.precision, dense=args.dense)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        ctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, wl.gamma, wl.block, opts, stream=stream)
        V0 = torch.from_numpy(si.start_block(p.n, wl.block, wl.seed)).cuda()
        found = []
        last = None
        for _ in range(args.warmup):
            last = ctx.solve(V0)
        stream.synchronize()

        def barrier():
            if world > 1:
                torch.distributed.barrier()
            torch.cuda.synchronize()

        barrier()
        cp, cf = clocks_start(args.clocks_csv)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        stats = []
        e0.record(stream)
        for _ in range(args.steps):
            rc, nf, ev, X, rs, st = ctx.solve(V0)
            found.append(nf)
            stats.append(st)
            last = (rc, nf, ev, X, rs, st)
        e1.record(stream)
        barrier()
        clk = clocks_stop(cp, cf, local)
        ms = e0.elapsed_time(e1)
        total_found, ms_max = reduce_over_ranks(sum(found), ms, world)
        rc, nf, ev, X, rs, st = last
        maxres = float(rs.max().item())
        # kernel-level roofline of the dominant kernel (the fused shifted SpMM + COCG phase 1)
        tim = ctx.filter_timing(V0[:, :wl.block])
        # end-to-end through the host-buffer entry point
        pin = lambda a: torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()
        hrp, hcol, hA, hB = pin(p.rowptr), pin(p.col.astype(np.int32)), pin(p.valA), pin(p.valB)
        hV0 = pin(si.start_block(p.n, wl.block, wl.seed))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev_h, X_h, rs_h, st_h = slrf.slrf_solve_host(hrp, hcol, hA, hB, wl.gamma, wl.block, opts, hV0)
        e2e_s = time.perf_counter() - t0
        h2d = hrp.nbytes + hcol.nbytes + hA.nbytes + hB.nbytes + hV0.nbytes
        d2h = ev_h.nbytes * 2 + p.n * wl.block * 8
        mixed = None
        if args.precision == 0 and args.mixed_it_max > 0:
            # the same workload with complex-FP32 inner solves inside the FP64 outer loop
            mopts = slrf.slrf_opts_default(m=wl.m, it_max=args.mixed_it_max, precision=1)
            mctx = slrf.Context(p.rowptr, p.col, p.valA, p.valB, wl.gamma, wl.block, mopts, stream=stream)
            for _ in range(args.warmup):
                mctx.solve(V0)
            barrier()
            m0 = torch.cuda.Event(enable_timing=True)
            m1 = torch.cuda.Event(enable_timing=True)
            mfound = []
            m0.record(stream)
            for _ in range(args.steps):
                mres = mctx.solve(V0)
                mfound.append(mres[1])
            m1.record(stream)
            barrier()
            mms = m0.elapsed_time(m1)
            mev = mres[2].cpu().numpy()
            fev = ev.cpu().numpy()
            dev_ = float(np.max(np.abs(mev - fev) / fev)) if len(mev) == len(fev) else None
            mtot, mms = reduce_over_ranks(sum(mfound), mms, world)
            mixed = {"value": mtot / (mms / 1e3), "unit": "eigenpairs/s", "it_max": args.mixed_it_max,
                     "ms_per_step": mms / args.steps, "eigenpairs_found": mres[1],
                     "max_resid": float(mres[4].max().item()),
                     "max_rel_eig_diff_vs_fp64": dev_, "outer_iters": mres[5]["outer_iters"],
                     "ms_filter_per_step": mres[5]["ms_filter"], "ms_dense_per_step": mres[5]["ms_dense"]}
            mctx.close()

    value = total_found / (ms_max / 1e3)
    col_solves = sum(s["column_solves"] for s in stats)
    col_iters = sum(s["column_iterations"] for s in stats)
    launches = sum(s["kernel_launches"] for s in stats)
    k0 = wl.block
    nnz, n, m = p.nnz, p.n, wl.m
    elem = 16 if args.precision == 0 else 8
    flops_spmm = 8.0 * nnz * m * k0 + 32.0 * n * m * k0
    bytes_spmm = elem * n * m * k0 * 5 + nnz * (4 + 2 * (8 if args.precision == 0 else 4))
    spmm_ms = tim["ms_spmm"] / max(tim["n_spmm"], 1)
    if args.precision == 0:
        achieved = flops_spmm / (spmm_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS,
                "traffic": SPMM64_TRAFFIC_Q1_41 if (args.workload == "q1_lap_41" and k0 == 160 and m == 8) else None,
                "kernel": "cocg_spmm_kernel<double>",
                "note": ("FP64 FMA pipe bound: 8 flops/nnz/complex column + 32 flops/row/column per launch; "
                         "peak = 152 SMs x 2 FP64 FMA/clk x 2 x 2.07 GHz (measured 1.197 TFLOP/s at 1.98 GHz)"),
                "hbm_gbs_algorithmic": bytes_spmm / (spmm_ms / 1e3) / 1e9}
    else:
        peak = 6701.5
        achieved = bytes_spmm / (spmm_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": None, "kernel": "cocg_spmm_kernel<float>", "note": "of measured hbm_gbs"}
    line = {
        "metric": METRIC, "value": value, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == 0 else "c32-in-f64",
        "data": "synthetic",
        "config": {"workload": f"{args.workload}: {desc}", "it_max": wl.it_max, "precision": args.precision,
                   "l2": "inputs larger than L2 (COCG state %.1f GB)" % (4 * elem * n * m * k0 / 1e9),
                   "parallelism": f"replicas x{world}"},
        "column_solves_per_s": col_solves * world / (ms_max / 1e3),
        "column_iterations_per_s": col_iters * world / (ms_max / 1e3),
        "spmm_gbs_algorithmic": bytes_spmm / (spmm_ms / 1e3) / 1e9,
        "eigenpairs_found": nf, "max_resid": maxres, "outer_iters": st["outer_iters"],
        "ms_filter_per_step": sum(s["ms_filter"] for s in stats) / args.steps,
        "ms_dense_per_step": sum(s["ms_dense"] for s in stats) / args.steps,
        "roofline": roof,
        "e2e": {"value": len(ev_h) / e2e_s, "unit": "eigenpairs/s", "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(launches),
        "clocks": clk,
        "mixed_precision": mixed,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_subprocess(args.workload, wl.it_max, nf, int(col_iters / args.steps),
                                                       st["outer_iters"])
    if rank == 0:
        print(json.dumps(line))
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()


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


def cpu_baseline_subprocess(name, it_max, n_found, col_iters, outer):
    code = ("import json,sys; sys.path.insert(0, %r); import bench; "
            "print(json.dumps(bench.cpu_baseline_sample(%r, %d, %d, %d, %d)))" %
            (ROOT, name, it_max, n_found, col_iters, outer))
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, env=env, timeout=600)
    try:
        return json.loads(r.stdout.strip().splitlines()[-1])
    except Exception:
        return {"value": None, "error": r.stderr[-300:]}


def reference_arm(args, rank, world):
    """The oracle as it stands on the host cores, same workload, metric and unit.  Each step
    is a bounded sample (cpu_baseline_sample) scaled to one whole solve with the workload's
    recorded solve counts.  Under torchrun only rank 0 works."""
    if rank != 0:
        return
    wl, desc = workload(args.workload, args.it_max)
    cnt = SOLVE_COUNTS.get(args.workload)
    if cnt is None:
        print(json.dumps({"impl": "reference", "unavailable": f"no recorded solve counts for {args.workload}"}))
        return
    vals = []
    t_start = time.perf_counter()
    for s in range(args.warmup + args.steps):
        r = cpu_baseline_sample(args.workload, wl.it_max, cnt["n_found"], cnt["column_iterations"], cnt["outer"],
                                budget_s=8.0)
        if s >= args.warmup:
            vals.append(r)
    v = statistics.median([r["value"] for r in vals])
    line = {"metric": METRIC, "value": v, "unit": "eigenpairs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": (time.perf_counter() - t_start) * 1e3 / (args.warmup + args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {desc}", "it_max": wl.it_max, "precision": 0},
            "impl": "reference",
            "cpu_baseline": {"value": v, "unit": "eigenpairs/s", "cores": 1, "kind": "oracle",
                             "sample": vals[-1]["sample"]},
            "e2e": {"value": v, "unit": "eigenpairs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))


if __name__ == "__main__":
    main()
