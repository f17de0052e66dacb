#!/usr/bin/env python
"""Benchmark of the GB300 HEVI 1D-IMEX library.

Workload (the GPU-scale configuration): 96 x 96 x 12 spectral elements of order N = 4 over a
200 x 200 x 15 km box (385 x 385 columns of 49 levels, 7,263,025 nodes), FP64, isentropic
reference state theta0 = 300 K plus a seeded 8-mode theta' perturbation (balanced rho').

A timed "step" is one HEVI 1D-IMEX ARK2 step at vertical Courant number C = 15
(dt = 9.32 s): three explicit right-hand sides, two fused implicit stages (predictor,
Schur right-hand side, stored-LU column solve, extraction) and the final update.  Every
timed step advances the same resident input state to a separate output buffer, so the
(horizontally unstable, C_H = 9) configuration never overflows during timing; the state
(290 MB) and the stored factors (0.99 GB) are larger than L2, so no L2 flush is needed.

value = simulated seconds per wall-clock second of that step (dt / step time).  Measured
alongside, outside the headline timed region: 1D-IMEX at C = 150 and the explicit RK35
comparator at C = 1, and their sim-s/wall-s ratios; the per-kernel algorithmic bytes and
HBM fractions (`kernels`), the FP64 roofline of the dominant kernel (`roofline`), the
stand-alone column solve against the HBM roofline (`column_solve`), the end-to-end figure
through host buffers (`e2e`), the accuracy of the C = 15 and C = 150 runs against RK35 at
C = 1 (`accuracy_vs_explicit_c1`), the speed-up at a stated accuracy for 1D- and 3D-IMEX
(`matched_accuracy`), 3D-IMEX on the headline box and at large aspect ratio (`imex3d`,
`imex3d_large_aspect`), and one entry per form and variant.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

--impl reference times the FP64 NumPy oracle on the host cores over the whole workload: one
single-threaded process per core, each advancing its block of columns (with a halo that
makes its owned nodes exact) by the same ARK2 steps; the time per step is the slowest
process's (oracle_partitioned).
"""
import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import time

if "reference" in sys.argv:
    # the oracle arm runs single-threaded: fix the BLAS thread count before numpy loads
    for _v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[_v] = "1"

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

NEX = NEY = 96
NEZ = 12
N = 4
LX = LY = 200e3
LZ = 15e3
C_MAIN = 15.0
SEED = 2024
GAMMA = 1004.67 / (1004.67 - 287.17)
C_S = (GAMMA * 287.17 * 300.0) ** 0.5          # sound speed at theta0 = 300 K
FP64_PEAK_TFLOPS = 152 * 4 * 2.07e9 / 1e12      # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz


def hbm_peak():
    """(GB/s, source): the measured copy bandwidth of this GPU pool when its record is
    present, else the earlier GB300 measurement of 6800 GB/s."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"
METRIC = "1D-IMEX sim-seconds/wall-second vs explicit C=1 on 1 GB300; % of HBM roofline"
WORKLOAD = ("96x96x12 hex elements over 200x200x15 km, N=4 (385x385 columns x 49 levels), FP64, "
            "HEVI 1D-IMEX ARK2 step at C=15")


def lgl_min_fraction(n):
    """Smallest LGL spacing on [-1, 1] / 2 (first interior node), for the Courant number."""
    c = np.zeros(n + 1)
    c[n] = 1.0
    r = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)).real)
    return (r[0] + 1.0) / 2.0


def dt_for(C):
    dz_min = lgl_min_fraction(N) * (LZ / NEZ)
    return C * dz_min / C_S


def dx_min():
    return lgl_min_fraction(N) * (LX / NEX)


def rhs_flops_per_node():
    """Algorithmic FP64 flops of one right-hand side per global node: 18 derivative dot
    products of length N+1 (2(N+1) flops each) and the pointwise Set2NC tendencies (46)."""
    return 18 * 2 * (N + 1) + 46


def envelope_entries(n=N, nez=NEZ):
    """Nonzero factor entries of one column's Schur-form LU (the envelope of S, pattern of
    D_z^2): column j of L holds 2N - r entries below the diagonal, column j of U N + r
    above it (r = j mod N; 2N at interfaces), cut at the column ends.  Returns (L, U with
    its diagonal)."""
    M = nez * n + 1
    nl = sum(min(2 * n if j % n == 0 else 2 * n - j % n, M - 1 - j) for j in range(M))
    nu = sum(min(2 * n if j % n == 0 else n + j % n, j) + 1 for j in range(M))
    return nl, nu


def solve_fma_per_unknown(n=N, nez=NEZ):
    """FP64 multiply-adds per unknown of the two substitutions over the envelope (the
    off-diagonal entries, plus one multiply by the inverted pivot)."""
    nl, nu = envelope_entries(n, nez)
    return (nl + nu) / (nez * n + 1)


def stage_flops_per_node(stage):
    """Algorithmic flops of one fused implicit stage per node (predictor, Schur RHS with a
    length-(2N+1) vertical derivative, banded solve over the factors' envelope,
    extraction)."""
    pred = (3 * 4 + 2 * 2) if stage == 3 else (3 * 2 + 2 * 1)
    schur = 4 + 2 * (N + 1) + 4
    solve = 2 * solve_fma_per_unknown()
    extract = 2 * (N + 1) + 8
    recomb = 2 * 3 if stage == 3 else 3
    return 2 * pred + schur + solve + extract + recomb


def alg_bytes_per_node(kernel, hb=2 * N):
    """Algorithmic HBM bytes per global node and launch, averaged over one ARK2 step.
    k_rhs: the five state fields and P' read, five tendencies (or the updated state)
    written.  k_pressure: rho' and theta' read, P' written.  k_stage (mean of stages 2 and
    3): q^n and R1 (stage 3 also R2 and q(2)) read, the envelope's factor entries read
    (envelope_entries per column over M unknowns), the stage value and its P' written."""
    if kernel == "k_rhs":
        return 8 * (6 + 5)
    if kernel == "k_pressure":
        return 8 * (2 + 1)
    fac = solve_fma_per_unknown()
    return 8 * (0.5 * ((5 + 5) + (5 + 5 + 5 + 5)) + fac + 6)


def source_sha(*names):
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_1702_04316_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:12]


def recorded_traffic(kernel, sha):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this source."""
    path = os.path.join(ROOT, "profiles", "%s_full_size.md" % kernel)
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)\s+source_sha:\s*([0-9a-f]+)", txt)
    if not m or m.group(2) != sha:
        return None
    return float(m.group(1))


# ---------------------------------------------------------------------------------------
def make_state(levels, xg, yg, zg, amp=0.5):
    import synthetic
    return synthetic.balanced_state(xg, yg, zg, LX, LY, LZ, levels["rho0"], levels["theta0"],
                                    SEED, amp)


def axis_coords(ne, h, xi):
    c = np.empty(ne * N + 1)
    for e in range(ne):
        c[e * N:e * N + N + 1] = e * h + (1.0 + xi) * h / 2.0
    return c


def lgl_nodes():
    c = np.zeros(N + 1)
    c[N] = 1.0
    r = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)).real)
    return np.concatenate([[-1.0], r, [1.0]])


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device):
        self.device = device
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.device), "--query-gpu=" + self.Q,
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            out, _ = self.p.communicate(timeout=5)
        except Exception:
            self.p.kill()
            out = ""
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": float(max(mx)) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


# ---------------------------------------------------------------------------------------
def measured_fp64_gemm_tflops(torch, n=4096, reps=5):
    """Best-of-reps FP64 GEMM rate (torch.matmul, a library GEMM) on the current GPU."""
    a = torch.randn(n, n, dtype=torch.float64, device="cuda")
    b = torch.randn(n, n, dtype=torch.float64, device="cuda")
    c = torch.empty_like(a)
    torch.matmul(a, b, out=c)
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        torch.matmul(a, b, out=c)
        e1.record()
        e1.synchronize()
        best = min(best, e0.elapsed_time(e1))
    del a, b, c
    return 2.0 * n ** 3 / (best * 1e-3) / 1e12


def max_over_ranks(x, dist, device):
    """The largest value of x over the ranks of the job (x itself when running alone)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(dt, ms_step, world):
    """Whole-job sim-s/wall-s of `world` independent replicas whose slowest step took
    ms_step: the simulated time all of them advanced, over that wall time."""
    return dt / (ms_step / 1e3) * world


def run_gpu_partitioned(args, world, rank, local, dist):
    """N > 1 GPUs: the workload split over a px x py process grid (strong scaling), each rank
    stepping its window with the phased step and a halo exchange over NCCL before every
    right-hand side (paper_1702_04316_gb300.partition).  value: the whole mesh's simulated
    seconds per wall second, timed as the slowest rank's."""
    import torch
    import paper_1702_04316_gb300 as pkg
    from paper_1702_04316_gb300.partition import PartitionedHEVI, process_grid
    dev = torch.device("cuda", local)
    px, py = process_grid(world)
    dt15 = dt_for(C_MAIN)
    part = PartitionedHEVI(NEX, NEY, NEZ, LX, LY, LZ, N, dt15, px, py, rank, dist=dist, device=dev)
    lev = part.ctx.reference_levels()
    xi = lgl_nodes()
    # this window's part of the global state (the halo already holds the owners' values)
    qg = make_state(lev, axis_coords(NEX, LX / NEX, xi), axis_coords(NEY, LY / NEY, xi), lev["z"])
    q0h = part.restrict(qg)
    del qg
    q0 = torch.from_numpy(q0h).to(dev)
    q1 = torch.empty_like(q0)
    stream = torch.cuda.current_stream()

    def time_steps(fn, k):
        dist.barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        b.synchronize()
        torch.cuda.synchronize()
        dist.barrier()
        return max_over_ranks(a.elapsed_time(b), dist, dev)

    step = lambda: part.step(q0, q1, 1)
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms = time_steps(step, args.steps)
    clk = clocks.stop()
    ms_step = ms / args.steps
    assert part.ctx.count_nonfinite(q1) == 0, "non-finite output"
    assert part.ctx.status() == pkg.NUMA_OK
    # end to end: this rank's window from pinned host memory, the step, its window back
    qin = torch.from_numpy(q0h).pin_memory()
    qout = torch.empty_like(qin).pin_memory()

    def e2e_step():
        q0.copy_(qin, non_blocking=True)
        part.step(q0, q1, 1)
        qout.copy_(q1, non_blocking=True)
        torch.cuda.current_stream().synchronize()
    for _ in range(max(3, args.warmup)):
        e2e_step()
    dist.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)
    nbytes = q0.numel() * 8
    out = {
        "metric": METRIC, "value": round(dt15 / (ms_step / 1e3), 3), "unit": "sim-s/wall-s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "C_V": C_MAIN, "dt_s": round(dt15, 5),
                   "columns": (NEX * N + 1) * (NEY * N + 1), "levels": NEZ * N + 1,
                   "l2": "inputs larger than L2; no flush",
                   "parallelism": "%d x %d horizontal partition, halo exchange over NCCL before "
                                  "every right-hand side" % (px, py)},
        "e2e": {"value": round(dt15 * args.steps / e2e_s, 3), "unit": "sim-s/wall-s",
                "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes,
                "api": "PartitionedHEVI.step (each rank's window from pinned host buffers)"},
        # per step: pre-pass, 3 right-hand sides, 2 stages, and a gather and a scatter per
        # neighbour at each of the 3 exchanges (rank 0's count)
        "gpu_launches": (6 + 6 * len(part.halo.peers)) * args.steps,
        "clocks": clk,
    }
    part.close()
    if rank == 0:
        print(json.dumps(out))
    dist.barrier()
    dist.destroy_process_group()


def run_gpu(args):
    import torch
    import paper_1702_04316_gb300 as pkg

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    if world > 1:
        return run_gpu_partitioned(args, world, rank, local, dist)
    dev = torch.device("cuda", local)

    dt15, dt150, dt1 = dt_for(C_MAIN), dt_for(150.0), dt_for(1.0)
    g = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dt15)
    lev = g.reference_levels()
    xi = lgl_nodes()
    xg = axis_coords(NEX, LX / NEX, xi)
    yg = axis_coords(NEY, LY / NEY, xi)
    q0h = make_state(lev, xg, yg, lev["z"])
    q0 = torch.from_numpy(q0h).to(dev)
    q1 = torch.empty_like(q0)
    nbytes_state = q0.numel() * 8

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.current_stream()

    def time_steps(fn, k):
        barrier()
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(k):
            fn()
        b.record(stream)
        b.synchronize()
        torch.cuda.synchronize()
        barrier()
        return max_over_ranks(a.elapsed_time(b), dist, dev)

    imex = lambda: g.step_imex1d(q0, q1, 1)
    for _ in range(args.warmup):
        imex()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    g.profile(True)
    ms = time_steps(imex, args.steps)
    g.profile(False)
    clk = clocks.stop()
    kt = {k: g.profile_read(k) for k in (pkg.K_PRESSURE, pkg.K_RHS, pkg.K_STAGE)}
    ms_step = ms / args.steps
    value = replica_value(dt15, ms_step, world)
    assert g.count_nonfinite(q1) == 0, "non-finite output"
    assert g.status() == pkg.NUMA_OK

    # C = 150: same kernels, different factors
    g150 = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dt150)
    for _ in range(args.warmup):
        g150.step_imex1d(q0, q1, 1)
    ms150 = time_steps(lambda: g150.step_imex1d(q0, q1, 1), args.steps) / args.steps
    g150.close()
    # explicit RK35 at C = 1
    rk = lambda: g.step_explicit_rk(q0, dt1, q1, 1)
    for _ in range(args.warmup):
        rk()
    ms_rk = time_steps(rk, args.steps) / args.steps
    sps = lambda dt, m: dt / (m / 1e3)

    # end to end through the host-buffer entry point: H2D of the state, the step, D2H
    qin = torch.from_numpy(q0h).pin_memory()
    qout = torch.empty_like(qin).pin_memory()
    for _ in range(max(3, args.warmup)):
        g.run_host(0, qin, 1, 0.0, qout)
    barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        g.run_host(0, qin, 1, 0.0, qout)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dist, dev)

    # roofline of the dominant kernel (by measured share of the step)
    nnode = g.nnode
    shares = {k: v[0] for k, v in kt.items()}
    names = {pkg.K_PRESSURE: "k_pressure", pkg.K_RHS: "k_rhs", pkg.K_STAGE: "k_stage"}
    srcs = {pkg.K_PRESSURE: ("rhs.cu", "rhs_device.cuh"), pkg.K_RHS: ("rhs.cu", "rhs_device.cuh"),
            pkg.K_STAGE: ("column.cu", "column_device.cuh")}
    top = max(shares, key=shares.get)
    tot_ms, launches = kt[top]
    per_launch_ms = tot_ms / max(launches, 1)
    if top == pkg.K_RHS:
        flops = rhs_flops_per_node() * nnode
    elif top == pkg.K_STAGE:
        flops = 0.5 * (stage_flops_per_node(2) + stage_flops_per_node(3)) * nnode
    else:
        flops = 40 * nnode
    achieved = flops / (per_launch_ms / 1e3) / 1e12
    sha = source_sha(*srcs[top], "numa_internal.cuh")
    traffic = recorded_traffic(names[top], sha)
    roofline = {"bound": "alu", "achieved": round(achieved, 4), "peak": round(FP64_PEAK_TFLOPS, 4),
                "unit": "TFLOP/s", "frac": round(achieved / FP64_PEAK_TFLOPS, 4), "traffic": traffic,
                "kernel": names[top], "per_launch_ms": round(per_launch_ms, 4),
                "peak_note": "FP64 FMA peak: 152 SMs x 2 FMA/clk x 2 flop x 2.07 GHz (unit counts x max clock)"}
    # context for the derived peak: what a library FP64 GEMM reaches on this GPU (the FP64 pipe
    # and the FP64 tensor cores run at about the same rate here)
    fp64_gemm = measured_fp64_gemm_tflops(torch)
    roofline["measured_fp64_gemm_tflops"] = round(fp64_gemm, 4)
    roofline["frac_of_measured_fp64_gemm"] = round(achieved / fp64_gemm, 4)
    hbm, hbm_src = hbm_peak()
    kernel_ms = {}
    for k, v in kt.items():
        per = v[0] / max(v[1], 1)
        gbs = alg_bytes_per_node(names[k]) * nnode / (per * 1e-3) / 1e9
        kernel_ms[names[k]] = {"total_ms": round(v[0], 3), "launches": v[1],
                               "share": round(v[0] / max(ms, 1e-9), 4),
                               "alg_bytes_per_node": alg_bytes_per_node(names[k]),
                               "achieved_gbs": round(gbs, 1),
                               "frac_of_hbm_peak": round(gbs / hbm, 4)}

    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "sim-s/wall-s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOAD, "C_V": C_MAIN, "C_H": round(C_S * dt15 / dx_min(), 3),
                   "dt_s": round(dt15, 5), "columns": g.ncol, "levels": g.M, "nodes": nnode,
                   "l2": "inputs larger than L2 (state 290 MB, factors 0.99 GB); no flush",
                   "parallelism": "replicas" if world > 1 else "single GPU"},
        "imex_c15": {"sim_s_per_wall_s": round(sps(dt15, ms_step), 3), "ms_per_step": round(ms_step, 4),
                     "dt_s": round(dt15, 5)},
        "imex_c150": {"sim_s_per_wall_s": round(sps(dt150, ms150), 3), "ms_per_step": round(ms150, 4),
                      "dt_s": round(dt150, 5), "C_H": round(C_S * dt150 / dx_min(), 2)},
        "explicit_c1": {"sim_s_per_wall_s": round(sps(dt1, ms_rk), 3), "ms_per_step": round(ms_rk, 4),
                        "dt_s": round(dt1, 5), "scheme": "RK35 (5-stage 3rd-order SSP)"},
        "speedup_vs_explicit_c1": {"C15": round(sps(dt15, ms_step) / sps(dt1, ms_rk), 3),
                                   "C150": round(sps(dt150, ms150) / sps(dt1, ms_rk), 3)},
        "e2e": {"value": round(dt15 * args.steps / e2e_s * world, 3), "unit": "sim-s/wall-s",
                "h2d_bytes_per_step": nbytes_state, "d2h_bytes_per_step": nbytes_state,
                "api": "numa_run_host (pinned host buffers, one step per call)"},
        "roofline": roofline,
        "kernels": kernel_ms,
        "gpu_launches": int(sum(v[1] for v in kt.values())),
        "clocks": clk,
    }
    # the standalone column solve (numa_solve_columns, step a4) against the HBM roofline:
    # algorithmic bytes = the stored factors + the right-hand side read + the solution written
    fb = g.query(pkg.Q_FACTOR_BYTES)
    nn = g.query(pkg.Q_NNODE)
    bcol = torch.randn(nn, dtype=torch.float64, device="cuda")
    xcol = torch.empty_like(bcol)
    for _ in range(args.warmup):
        g.solve_columns(bcol, xcol)
    ms_solve = time_steps(lambda: g.solve_columns(bcol, xcol), args.steps) / args.steps
    # algorithmic bytes: the factors' envelope (the stored band beyond it is exact zeros and
    # is not read), the right-hand side and the solution
    nl, nu = envelope_entries()
    solve_bytes = 8 * (nl + nu) * g.ncol + 2 * 8 * nn
    fma = solve_fma_per_unknown()
    out["column_solve"] = {"ms_per_launch": round(ms_solve, 4), "bytes_per_launch": int(solve_bytes),
                           "stored_factor_bytes": int(fb),
                           "achieved_gbs": round(solve_bytes / (ms_solve * 1e-3) / 1e9, 1),
                           "hbm_peak_gbs": hbm, "peak_source": hbm_src,
                           "frac_of_hbm_peak": round(solve_bytes / (ms_solve * 1e-3) / 1e9 / hbm, 4),
                           "fp64_floor_ms": round(fma * nn / (FP64_PEAK_TFLOPS * 1e12 / 2) * 1e3, 4),
                           "note": "%.2f FP64 multiply-adds per unknown (L and U substitutions over "
                                   "the factors' envelope)" % fma}
    del bcol, xcol
    # the mixed-precision form on the same workload
    gm = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dt15, precision="mixed", refine_iters=1)
    for _ in range(args.warmup):
        gm.step_imex1d(q0, q1, 1)
    ms_mx = time_steps(lambda: gm.step_imex1d(q0, q1, 1), args.steps) / args.steps
    gm.close()
    out["imex_c15_mixed"] = {"sim_s_per_wall_s": round(sps(dt15, ms_mx), 3), "ms_per_step": round(ms_mx, 4),
                             "form": "FP32 RHS over FP64 reference, FP32 LU + 1 FP64 refinement sweep"}
    g32 = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dt15, precision="rhs32")
    for _ in range(args.warmup):
        g32.step_imex1d(q0, q1, 1)
    ms_32 = time_steps(lambda: g32.step_imex1d(q0, q1, 1), args.steps) / args.steps
    g32.close()
    out["imex_c15_rhs32"] = {"sim_s_per_wall_s": round(sps(dt15, ms_32), 3), "ms_per_step": round(ms_32, 4),
                             "form": "FP32 RHS over FP64 reference, FP64 column LU"}
    gdf = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dt15, precision="df")
    for _ in range(args.warmup):
        gdf.step_imex1d(q0, q1, 1)
    ms_df = time_steps(lambda: gdf.step_imex1d(q0, q1, 1), args.steps) / args.steps
    gdf.profile(True)
    gdf.step_imex1d(q0, q1, 1)
    t_df, n_df = gdf.profile_read(pkg.K_RHS)
    t_pd, n_pd = gdf.profile_read(pkg.K_PRESSURE)
    gdf.profile(False)
    r64 = g.rhs_explicit(q0)
    rdf = gdf.rhs_explicit(q0)
    # relative L2 per field; a field whose FP64 tendency is exactly zero (rho' and theta' of
    # a balanced state at rest) reports its absolute L2 relative to the largest field norm
    scale = max(float(torch.linalg.norm(r64[f])) for f in range(5))
    rel = [float(torch.linalg.norm(rdf[f] - r64[f])) / (float(torch.linalg.norm(r64[f])) or scale or 1.0)
           for f in range(5)]
    gdf.close()
    out["imex_c15_df"] = {"sim_s_per_wall_s": round(sps(dt15, ms_df), 3), "ms_per_step": round(ms_df, 4),
                          "rhs_ms_per_launch": round(t_df / max(n_df, 1), 4),
                          "prepass_ms_per_launch": round(t_pd / max(n_pd, 1), 4),
                          "rhs_rel_l2_vs_fp64_kernel": [float("%.3g" % x) for x in rel],
                          "form": "double-float (FP32-pair) derivative sums and pointwise products "
                                  "in the RHS; FP64 EOS, column LU and state"}
    # the higher-order schemes on the same workload: ARK3(2)4L[2]SA (4 RHS + 3 column stages
    # per step), ARK4(3)6L[2]SA (6 + 5, general fused stage), ARK5(4)8L[2]SA (8 + 7)
    for scheme, name in (("ark3", "ARK3(2)4L[2]SA"), ("ark4", "ARK4(3)6L[2]SA"),
                         ("ark5", "ARK5(4)8L[2]SA")):
        res = {}
        for C, dtc in ((15, dt15), (150, dt150)):
            gs = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dtc, scheme=scheme)
            for _ in range(args.warmup):
                gs.step_imex1d(q0, q1, 1)
            mss = time_steps(lambda: gs.step_imex1d(q0, q1, 1), args.steps) / args.steps
            gs.profile(True)
            gs.step_imex1d(q0, q1, 1)
            t_st, n_st = gs.profile_read(pkg.K_STAGE)
            gs.profile(False)
            gs.close()
            res["C%d" % C] = {"sim_s_per_wall_s": round(sps(dtc, mss), 3), "ms_per_step": round(mss, 4),
                              "stage_ms_per_launch": round(t_st / max(n_st, 1), 4),
                              "speedup_vs_explicit_c1": round(sps(dtc, mss) / sps(dt1, ms_rk), 3)}
        out["imex_" + scheme] = dict(res, scheme=name + ", FP64, Schur form")
    if not args.no_forms:
        out["imex3d"] = imex3d_form(pkg, torch, q0, ms_rk, args.warmup)
        out["imex3d_large_aspect"] = imex3d_aspect_form(pkg, torch, ms_rk)
    if not args.no_forms:
        out["accuracy_vs_explicit_c1"] = accuracy_vs_explicit(pkg, torch)
        out["matched_accuracy"] = matched_accuracy(pkg, torch, ms_rk,
                                                   {"fp64": ms_step, "rhs32": ms_32})
        out["precision_form"] = precision_form(pkg, torch, min(args.steps, 20), args.warmup)
        out["batching_form"] = batching_form(pkg, torch, min(args.steps, 10), args.warmup)
        out["batching_form_small_members"] = batching_form(pkg, torch, min(args.steps, 20), args.warmup,
                                                           64, (8, 8), (6, 6), (4, 4), 4500)
        out["differentiation_form"] = differentiation_form(pkg, torch, args.warmup)
        out["column_forms"] = column_forms(pkg, torch, q0, min(args.steps, 10), args.warmup)
    if rank == 0 and not args.no_cpu_baseline:
        out["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
    g.close()
    if rank == 0:
        print(json.dumps(out))
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()


# ---------------------------------------------------------------------------------------
def accuracy_vs_explicit(pkg, torch, L=40000e3):
    """The accuracy at which the speedups over explicit RK35 at C = 1 hold.

    Same array shapes as the benchmark (96 x 96 x 12 elements, N = 4, 15 km deep, the same
    dt at each C_V and so the same cost per step), on a box stretched horizontally to
    L x L: on the 200 km box C_H = 0.6 C_V, and at C_V = 15 the explicit horizontal part is
    unstable (C_H = 9).  At L = 40,000 km C_H = 0.45 at C_V = 150, the paper's regime of
    large aspect ratio.  theta' is the benchmark's recipe (0.5 K) on the stretched box.
    Reference: RK35 at C = 1 to t = dt(C = 150) = 150 steps; its own error is estimated
    against RK35 at C = 0.5 (300 steps).  Relative L2 per field of 1D-IMEX ARK2 at C = 15
    (10 steps) and C = 150 (1 step), FP64 and the two FP32-RHS precision forms, against
    the reference."""
    dt1, dt15, dt150 = dt_for(1.0), dt_for(15.0), dt_for(150.0)
    g = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt15)
    lev = g.reference_levels()
    xi = lgl_nodes()
    import synthetic
    q0h = synthetic.balanced_state(axis_coords(NEX, L / NEX, xi), axis_coords(NEY, L / NEY, xi),
                                   lev["z"], L, L, LZ, lev["rho0"], lev["theta0"], SEED, 0.5)
    q0 = torch.from_numpy(q0h).cuda()
    names = ("rho", "u", "v", "w", "theta")

    def rel(a, b):
        out = {}
        for f, nm in enumerate(names):
            nb = float(torch.linalg.norm(b[f]))
            out[nm] = float("%.3g" % (float(torch.linalg.norm(a[f] - b[f])) / nb)) if nb > 0 else None
        return out

    ref = g.step_explicit_rk(q0, dt1, torch.empty_like(q0), 150)
    ref_half = g.step_explicit_rk(q0, 0.5 * dt1, torch.empty_like(q0), 300)
    res = {"box": "96x96x12 elements over %gx%g km x 15 km, N=4" % (L / 1e3, L / 1e3),
           "C_H_at_C_V_150": round(C_S * dt150 / (dx_min() * L / LX), 3),
           "t_s": round(dt150, 4),
           "reference": "RK35 at C=1 (150 steps)",
           "reference_vs_rk35_c0.5": rel(ref, ref_half)}
    res["imex_c15_fp64"] = rel(g.step_imex1d(q0, torch.empty_like(q0), 10), ref)
    g.close()
    g150 = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt150)
    res["imex_c150_fp64"] = rel(g150.step_imex1d(q0, torch.empty_like(q0), 1), ref)
    g150.close()
    for prec in ("mixed", "rhs32"):
        gp = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt15, precision=prec)
        res["imex_c15_" + prec] = rel(gp.step_imex1d(q0, torch.empty_like(q0), 10), ref)
        gp.close()
    res["batched"] = ("ensemble members are bitwise equal to single FP64 contexts, so their "
                      "accuracy is the FP64 form's")
    return res


MATCHED_C = (1, 2, 3, 5, 10, 15, 25, 30, 50, 75, 150)     # divisors of 150
MATCHED_BARS = {"theta": (1e-4, 1e-3), "w": (1e-2, 1e-1)}


def matched_accuracy(pkg, torch, ms_rk, ms_forms, L=40000e3):
    """Speed-up over explicit RK35 at C = 1 at a stated accuracy (the paper's 100X at
    C_V = 150 is a time to solution at matched results, Sec. "Acoustic wave problem").

    On the stretched box of accuracy_vs_explicit (same array shapes, so the same cost per
    step), 1D-IMEX ARK2 runs to t = dt(C = 150) at every C_V in MATCHED_C (150 / C steps);
    its relative L2 errors in theta' and w against RK35 at C = 1 (150 steps) are recorded.
    For each bar of MATCHED_BARS the largest C_V whose error stays under it is found, and
    the speed-up there is C_V x (RK35 ms per step) / (1D-IMEX ms per step), the step costs
    being those measured on the benchmark workload (ms_forms: form -> ms per step).  The
    ensemble form's members are bitwise the FP64 form's, so they share its accuracy.
    3D-IMEX (column-LU preconditioner) is run the same way; its cost per step depends on
    C_V, so each of its runs is timed on this machine."""
    dt1, dt150 = dt_for(1.0), dt_for(150.0)
    g1 = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt150)
    lev = g1.reference_levels()
    xi = lgl_nodes()
    import synthetic
    q0h = synthetic.balanced_state(axis_coords(NEX, L / NEX, xi), axis_coords(NEY, L / NEY, xi),
                                   lev["z"], L, L, LZ, lev["rho0"], lev["theta0"], SEED, 0.5)
    q0 = torch.from_numpy(q0h).cuda()
    ref = g1.step_explicit_rk(q0, dt1, torch.empty_like(q0), 150)
    ref_half = g1.step_explicit_rk(q0, 0.5 * dt1, torch.empty_like(q0), 300)
    g1.close()

    def rel(a, f):
        return float(torch.linalg.norm(a[f] - ref[f]) / torch.linalg.norm(ref[f]))
    res = {"box": "96x96x12 elements over %gx%g km x 15 km, N=4" % (L / 1e3, L / 1e3),
           "t_s": round(dt150, 4), "reference": "RK35 at C=1 (150 steps)",
           "reference_own_error_vs_rk35_c0.5": {"theta": float("%.3g" % rel(ref_half, 4)),
                                                "w": float("%.3g" % rel(ref_half, 3))},
           "rk35_ms_per_step": round(ms_rk, 4)}
    for form, ms_imex in ms_forms.items():
        errs = {}
        for C in MATCHED_C:
            gc = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt_for(float(C)),
                          precision="fp64" if form == "fp64" else form)
            out = gc.step_imex1d(q0, torch.empty_like(q0), 150 // C)
            errs[C] = (rel(out, 4), rel(out, 3))
            gc.close()
        entry = {"imex_ms_per_step": round(ms_imex, 4),
                 "errors": {"C%d" % C: {"theta": float("%.3g" % e[0]), "w": float("%.3g" % e[1])}
                            for C, e in errs.items()}}
        for fi, (nm, bars) in enumerate(MATCHED_BARS.items()):
            for bar in bars:
                ok = [C for C in MATCHED_C if errs[C][fi] <= bar]
                Cm = max(ok) if ok else None
                entry["%s<=%g" % (nm, bar)] = {
                    "largest_C_V": Cm,
                    "speedup_vs_explicit_c1": round(Cm * ms_rk / ms_imex, 2) if Cm else None}
        res[form] = entry
    # 3D-IMEX with the column-LU preconditioner: its cost per step grows with C_V (BiCGstab
    # iterations), so each C_V's run is timed (after one untimed step)
    errs, ms3d = {}, {}
    for C in MATCHED_C:
        gc = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt_for(float(C)), imex="3d", precond="column",
                      krylov_tol=1e-10, krylov_max_iters=4000)
        out = torch.empty_like(q0)
        gc.step_imex3d(q0, out, 1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        gc.step_imex3d(q0, out, 150 // C)
        e1.record()
        e1.synchronize()
        ms3d[C] = e0.elapsed_time(e1) / (150 // C)
        errs[C] = (rel(out, 4), rel(out, 3))
        gc.close()
    entry = {"imex_ms_per_step": {"C%d" % C: round(ms3d[C], 3) for C in MATCHED_C},
             "errors": {"C%d" % C: {"theta": float("%.3g" % e[0]), "w": float("%.3g" % e[1])}
                        for C, e in errs.items()}}
    for fi, (nm, bars) in enumerate(MATCHED_BARS.items()):
        for bar in bars:
            ok = [C for C in MATCHED_C if errs[C][fi] <= bar]
            Cm = max(ok) if ok else None
            entry["%s<=%g" % (nm, bar)] = {
                "largest_C_V": Cm,
                "speedup_vs_explicit_c1": round(Cm * ms_rk / ms3d[Cm], 2) if Cm else None}
    res["imex3d_column_lu"] = entry
    res["batched"] = "ensemble members are bitwise the FP64 form's: its entry applies"
    return res


# ---------------------------------------------------------------------------------------
def precision_form(pkg, torch, steps, warmup, nsteps_err=200):
    """The mixed-precision form on its own workload: 64 x 64 x 10 elements of order 7 over
    2000 x 2000 x 10 km (the box size is not given; this one keeps C_H = 0.48 at C_V = 15),
    seeded perturbation amplitude in [0.1, 2] K.  Times one HEVI step of each precision
    (out of place from the same input) and states the mixed form's relative L2 error of
    theta' and w after nsteps_err steps against the FP64 path."""
    import synthetic
    nex, nez, n, L, Lz, C = 64, 10, 7, 2000e3, 10e3, 15.0
    c = np.zeros(n + 1)
    c[n] = 1.0
    r = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)).real)
    xi = np.concatenate([[-1.0], r, [1.0]])
    fmin = (r[0] + 1.0) / 2.0
    dt = C * fmin * (Lz / nez) / C_S
    amp = float(np.random.Generator(np.random.PCG64(3000)).uniform(0.1, 2.0))
    out = {"workload": "64x64x10 hex elements over 2000x2000x10 km, N=7 (449x449 columns x 71 levels), "
                       "HEVI 1D-IMEX ARK2 at C=15",
           "dt_s": round(dt, 4), "C_H": round(C_S * dt / (fmin * L / nex), 3), "amp_K": round(amp, 4)}
    res = {}
    for prec in ("fp64", "mixed", "rhs32"):
        g = pkg.Numa(nex, nex, nez, L, L, Lz, n, dt, precision=prec, refine_iters=1)
        lev = g.reference_levels()
        h = L / nex
        ax = np.concatenate([e * h + (1.0 + xi[:-1]) * h / 2.0 for e in range(nex)] + [[L]])
        q0 = torch.from_numpy(synthetic.balanced_state(ax, ax, lev["z"], L, L, Lz, lev["rho0"],
                                                       lev["theta0"], 3001, amp)).cuda()
        q1 = torch.empty_like(q0)
        for _ in range(warmup):
            g.step_imex1d(q0, q1, 1)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(steps):
            g.step_imex1d(q0, q1, 1)
        b.record()
        b.synchronize()
        ms = a.elapsed_time(b) / steps
        qr = q0.clone()
        g.step_imex1d(qr, None, nsteps_err)
        torch.cuda.synchronize()
        res[prec] = (ms, qr, g.query(pkg.Q_FACTOR_BYTES))
        g.close()
    ms64, q64, fb64 = res["fp64"]
    msmx, qmx, fbmx = res["mixed"]
    ms32, q32, fb32 = res["rhs32"]
    def rel(f, q=None):
        q = qmx if q is None else q
        return float(torch.linalg.norm(q[f] - q64[f]) / torch.linalg.norm(q64[f]))
    out.update({
        "fp64": {"ms_per_step": round(ms64, 4), "sim_s_per_wall_s": round(dt / (ms64 / 1e3), 2),
                 "factor_bytes": fb64},
        "mixed": {"ms_per_step": round(msmx, 4), "sim_s_per_wall_s": round(dt / (msmx / 1e3), 2),
                  "factor_bytes": fbmx, "refine_iters": 1},
        "speedup_mixed_vs_fp64": round(ms64 / msmx, 3),
        "rel_l2_vs_fp64_after_%d_steps" % nsteps_err: {"theta": rel(4), "w": rel(3), "rho": rel(0)},
        "rhs32": {"ms_per_step": round(ms32, 4), "sim_s_per_wall_s": round(dt / (ms32 / 1e3), 2),
                  "factor_bytes": fb32, "speedup_vs_fp64": round(ms64 / ms32, 3),
                  "form": "FP32 RHS, FP64 column factors and solve",
                  "rel_l2_vs_fp64_after_%d_steps" % nsteps_err:
                      {"theta": rel(4, q32), "w": rel(3, q32), "rho": rel(0, q32)}},
        "finite": bool(torch.isfinite(qmx).all().item() and torch.isfinite(q64).all().item()
                       and torch.isfinite(q32).all().item()),
    })
    return out


def ensemble(pkg, torch, nmembers=64, h_range=(8, 48), v_range=(6, 16), n_range=(4, 6),
             seed=4000):
    """The batching form's seeded ensemble: nmembers members with uneven meshes (horizontal
    h_range x h_range elements, vertical v_range, order n_range), 50 km x 50 km elements over
    a 10 km depth, each at its own C = 15 time step, each with its own balanced perturbation
    of amplitude in [0.1, 2] K.  Returns (batch, state, meshes, orders, dts, nodes)."""
    import synthetic
    rng = np.random.Generator(np.random.PCG64(seed))
    meshes, Ns, dts, xis = [], [], [], {}
    for m in range(nmembers):
        nh = int(rng.integers(h_range[0], h_range[1] + 1))
        nz = int(rng.integers(v_range[0], v_range[1] + 1))
        n = int(rng.integers(n_range[0], n_range[1] + 1))
        meshes.append((nh, nh, nz, 50e3 * nh, 50e3 * nh, 10e3))
        Ns.append(n)
        c = np.zeros(n + 1)
        c[n] = 1.0
        r = np.sort(np.polynomial.legendre.legroots(np.polynomial.legendre.legder(c)).real)
        xis[n] = np.concatenate([[-1.0], r, [1.0]])
        dts.append(15.0 * (r[0] + 1.0) / 2.0 * (10e3 / nz) / C_S)
    b = pkg.Batch(meshes, Ns, dts)
    q = b.empty_state()
    nodes = 0
    for m, (mesh, n) in enumerate(zip(meshes, Ns)):
        nh, _, nz, L, _, Lz = mesh
        lev = b.reference_levels(m)
        h = L / nh
        xi = xis[n]
        ax = np.concatenate([e * h + (1.0 + xi[:-1]) * h / 2.0 for e in range(nh)] + [[L]])
        amp = float(rng.uniform(0.1, 2.0))
        st = synthetic.balanced_state(ax, ax, lev["z"], L, L, Lz, lev["rho0"], lev["theta0"], seed + 100 + m, amp)
        b.member(q, m).copy_(torch.from_numpy(st))
        nodes += st.shape[1]
    return b, q, meshes, Ns, dts, nodes


def batching_form(pkg, torch, steps, warmup, nmembers=64, h_range=(8, 48), v_range=(6, 16),
                  n_range=(4, 6), seed=4000):
    """Ensemble of nmembers independent members with seeded uneven meshes (horizontal 8x8 to
    48x48 elements, vertical 6-16, N = 4-6, FP64), each with its own seeded perturbation,
    advanced by HEVI 1D-IMEX at C = 15 (each member at its own dt).  Box sizes are not given:
    50 km x 50 km elements horizontally over a 10 km depth (C_H < 0.5).  Compares the
    ensemble path (persistent launches, CUDA graph per step, autotuned tiles) with stepping
    the members one context at a time."""
    b, q, meshes, Ns, dts, nodes = ensemble(pkg, torch, nmembers, h_range, v_range, n_range, seed)
    q1 = b.empty_state()
    for _ in range(warmup):
        b.step_imex1d(q, q1, 1)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        b.step_imex1d(q, q1, 1)
    e1.record()
    e1.synchronize()
    ms_batch = e0.elapsed_time(e1) / steps
    tuning = b.tuning()
    finite = bool(torch.isfinite(q1).all().item())
    # the same members, one context at a time
    ctxs = [pkg.Numa(*mesh[:3], *mesh[3:], n, dt) for mesh, n, dt in zip(meshes, Ns, dts)]
    views = [(b.member(q, m).contiguous(), torch.empty_like(b.member(q, m))) for m in range(nmembers)]
    def seq():
        for g, (a, o) in zip(ctxs, views):
            g.step_imex1d(a, o, 1)
    for _ in range(warmup):
        seq()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(steps):
        seq()
    e1.record()
    e1.synchronize()
    ms_seq = e0.elapsed_time(e1) / steps
    same = all(torch.equal(o, b.member(q1, m)) for m, (a, o) in enumerate(views))
    for g in ctxs:
        g.close()
    # the bound of the work itself: per order, the time per node-step of one large member
    # (48 x 48 x 12 elements, the biggest member shape, which fills the GPU), summed over the
    # ensemble's nodes of that order
    ns_node = {}
    for n in sorted(set(Ns)):
        nh, nz = 48, 12
        dtn = 15.0 * lgl_min_fraction(n) * (10e3 / nz) / C_S
        gb = pkg.Numa(nh, nh, nz, 50e3 * nh, 50e3 * nh, 10e3, n, dtn)
        qa = gb.empty_state().zero_()
        qb = gb.empty_state()
        for _ in range(warmup):
            gb.step_imex1d(qa, qb, 1)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            gb.step_imex1d(qa, qb, 1)
        e1.record()
        e1.synchronize()
        ns_node[n] = e0.elapsed_time(e1) / steps * 1e6 / gb.nnode
        gb.close()
    node_counts = {}
    for m, n in enumerate(Ns):
        node_counts[n] = node_counts.get(n, 0) + b.member_query(m, pkg.Q_NNODE)
    ms_bound = sum(node_counts[n] * ns_node[n] for n in node_counts) / 1e6
    b.close()
    sim = float(np.sum(dts))
    norders = len(set(Ns))
    return {"workload": "%d members, horizontal %d-%d elements, vertical %d-%d, N=%d-%d (seeded), C=15"
                        % ((nmembers,) + tuple(h_range) + tuple(v_range) + tuple(n_range)),
            "nodes": int(nodes), "members": nmembers,
            "ensemble": {"ms_per_step": round(ms_batch, 3),
                         "member_sim_s_per_wall_s": round(sim / (ms_batch / 1e3), 1),
                         "node_steps_per_s": float("%.4g" % (nodes / (ms_batch / 1e3))),
                         "launches_per_step": 1 + 5 * norders, "cuda_graph": True,
                         "autotuned": {str(k): v for k, v in tuning.items()}},
            "one_context_at_a_time": {"ms_per_step": round(ms_seq, 3),
                                      "launches_per_step": 8 * nmembers},
            "speedup": round(ms_seq / ms_batch, 3), "identical_to_single_contexts": same,
            "work_bound": {"ns_per_node_step_by_order": {str(k): round(v, 4) for k, v in ns_node.items()},
                           "nodes_by_order": {str(k): int(v) for k, v in node_counts.items()},
                           "ms_per_step": round(ms_bound, 3),
                           "ensemble_over_bound": round(ms_batch / ms_bound, 3),
                           "note": "each order's time per node-step in one 48x48x12-element "
                                   "context, summed over the ensemble's nodes of that order"},
            "finite": finite}


def column_forms(pkg, torch, q0, steps, warmup, nsteps_cmp=1):
    """The paper's memory / speed contrast of the two 1D column systems on the headline
    workload (96 x 96 x 12 elements, N = 4, C = 15): the Schur form (M x M, half-band 2N)
    and the standard form (3M x 3M on rho', w, theta', half-band 3N + 1), both FP64 with
    banded LU stored per column.  Times the factorisation and one HEVI step of each, and
    states how far the standard form's step is from the Schur form's (one step: this
    workload has C_H = 9, so longer runs do not stay bounded)."""
    dt = dt_for(C_MAIN)
    res = {}
    for form in ("schur", "standard"):
        g = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, 0.0, column_form=form)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        g.factor_columns(dt)
        e1.record()
        e1.synchronize()
        fact_ms = e0.elapsed_time(e1)
        q1 = torch.empty_like(q0)
        for _ in range(warmup):
            g.step_imex1d(q0, q1, 1)
        g.profile(True)
        torch.cuda.synchronize()
        e0.record()
        for _ in range(steps):
            g.step_imex1d(q0, q1, 1)
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        st_ms, st_n = g.profile_read(pkg.K_STAGE)
        g.profile(False)
        qr = q0.clone()
        g.step_imex1d(qr, None, nsteps_cmp)
        torch.cuda.synchronize()
        res[form] = {"factor_bytes": g.query(pkg.Q_FACTOR_BYTES), "half_band": g.query(pkg.Q_HALF_BAND),
                     "factor_ms": round(fact_ms, 3), "ms_per_step": round(ms, 4),
                     "sim_s_per_wall_s": round(dt / (ms / 1e3), 2),
                     "stage_ms_per_launch": round(st_ms / max(st_n, 1), 4)}, qr
        g.close()
    a, qa = res["schur"]
    b, qb = res["standard"]
    diff = {name: float(torch.linalg.norm(qb[f] - qa[f]) / torch.linalg.norm(qa[f]))
            for f, name in ((0, "rho"), (3, "w"), (4, "theta"))}
    return {"workload": "96x96x12 hex elements over 200x200x15 km, N=4 (385x385 columns x 49 levels), "
                        "HEVI 1D-IMEX ARK2 at C=15, FP64",
            "schur": a, "standard": b,
            "standard_over_schur": {"factor_bytes": round(b["factor_bytes"] / a["factor_bytes"], 3),
                                    "step_time": round(b["ms_per_step"] / a["ms_per_step"], 3),
                                    "stage_time": round(b["stage_ms_per_launch"] / a["stage_ms_per_launch"], 3)},
            "rel_l2_standard_vs_schur_after_%d_steps" % nsteps_cmp: diff}


def imex3d_form(pkg, torch, q0, ms_rk, warmup, steps=3):
    """3D-IMEX (Schur form, BiCGstab + Chebyshev polynomial preconditioner of degree P) on
    the headline workload, where C_H = 9 at C_V = 15 makes the horizontally explicit 1D-IMEX
    unstable and the 3D form (acoustics implicit in every direction) is the stable method.
    Per polynomial degree, and with the column-LU preconditioner: ms per step, BiCGstab
    iterations per step (two solves), the Schur operator's time per application and the
    speedup over explicit RK35 at C = 1."""
    out = {"workload": "96x96x12 hex elements over 200x200x15 km, N=4, FP64, ARK2, C_V=15 "
                       "(C_H=9), BiCGstab stop at 1e-10 preconditioned-residual drop"}
    dt = dt_for(C_MAIN)
    q1 = torch.empty_like(q0)
    for P in (1, 2, 4, "column"):
        kw = {"precond": "column"} if P == "column" else {"pbno_order": P}
        g = pkg.Numa(NEX, NEY, NEZ, LX, LY, LZ, N, dt, imex="3d", krylov_tol=1e-10,
                     krylov_max_iters=2000, **kw)
        for _ in range(max(1, warmup // 3)):
            g.step_imex3d(q0, q1, 1)
        g.profile(True)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        its = 0
        for _ in range(steps):
            g.step_imex3d(q0, q1, 1)
            its += g.imex3d_info()["iters_last_step"]
        e1.record()
        e1.synchronize()
        ms = e0.elapsed_time(e1) / steps
        t_s, n_s = g.profile_read(pkg.K_SCHUR3D)
        g.profile(False)
        info = g.imex3d_info()
        out["column_lu" if P == "column" else "P%d" % P] = {
                          "ms_per_step": round(ms, 3), "bicgstab_iters_per_step": its / steps,
                          "schur_op_ms_per_application": round(t_s / max(n_s, 1), 4),
                          "schur_op_applications_per_step": n_s / steps,
                          "l_max": round(info["l_max"], 3),
                          "sim_s_per_wall_s": round(dt / (ms / 1e3), 2),
                          "speedup_vs_explicit_c1": round((dt / ms) / (dt_for(1.0) / ms_rk), 3),
                          "finite": bool(torch.isfinite(q1).all().item())}
        g.close()
    return out


def stretched_state(pkg, torch, L):
    """The benchmark's balanced theta' recipe (0.5 K) on the box stretched to L x L."""
    import synthetic
    g = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, 0.0)
    lev = g.reference_levels()
    g.close()
    xi = lgl_nodes()
    q0h = synthetic.balanced_state(axis_coords(NEX, L / NEX, xi), axis_coords(NEY, L / NEY, xi),
                                   lev["z"], L, L, LZ, lev["rho0"], lev["theta0"], SEED, 0.5)
    return torch.from_numpy(q0h).cuda()


def imex3d_aspect_form(pkg, torch, ms_rk, steps=3, L=40000e3):
    """3D-IMEX in the paper's regime of large aspect ratio: the benchmark's array shapes on
    the box stretched to 40,000 x 40,000 km (C_H = 0.045 at C_V = 15, 0.45 at C_V = 150), where
    the vertical acoustics dominate the implicit operator.  Per preconditioner (Chebyshev of
    degree 1 and 4, column LU) and C_V: ms per step, BiCGstab iterations per step (two
    solves) and the speedup over explicit RK35 at C = 1, whose cost per step does not depend
    on the box's size."""
    q0 = stretched_state(pkg, torch, L)
    q1 = torch.empty_like(q0)
    out = {"workload": "96x96x12 hex elements over 40000x40000x15 km, N=4, FP64, ARK2, BiCGstab "
                       "stop at 1e-10 preconditioned-residual drop"}
    for C in (15, 150):
        dt = dt_for(float(C))
        res = {"C_H": round(C_S * dt / (dx_min() * L / LX), 3)}
        for P in (1, 4, "column"):
            kw = {"precond": "column"} if P == "column" else {"pbno_order": P}
            g = pkg.Numa(NEX, NEY, NEZ, L, L, LZ, N, dt, imex="3d", krylov_tol=1e-10,
                         krylov_max_iters=4000, **kw)
            g.step_imex3d(q0, q1, 1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            its = 0
            for _ in range(steps):
                g.step_imex3d(q0, q1, 1)
                its += g.imex3d_info()["iters_last_step"]
            e1.record()
            e1.synchronize()
            ms = e0.elapsed_time(e1) / steps
            res["column_lu" if P == "column" else "P%d" % P] = {
                "ms_per_step": round(ms, 3), "bicgstab_iters_per_step": its / steps,
                "speedup_vs_explicit_c1": round(C * ms_rk / ms, 2),
                "finite": bool(torch.isfinite(q1).all().item())}
            g.close()
        out["C%d" % C] = res
    return out


def differentiation_form(pkg, torch, warmup, reps=5, nsteps=20, every=5):
    """Gradient of J(q0) = 1/2 sum (theta'_T - target)^2 after nsteps HEVI 1D-IMEX steps at
    C = 15 on 16 x 16 x 8 elements of order 4 over 600 x 600 x 10 km (the box size is not
    given; this one keeps C_H = 0.5), FP64, checkpoints every `every` steps.  Times the
    checkpointed forward run, the adjoint sweep (segment recomputation included) and the
    tangent-linear run, reports the adjoint kernels' own times and checks the gradient by a
    dot-product test and by centred finite differences with step 1e-6."""
    import synthetic
    nex, nez, n, L, Lz, C = 16, 8, 4, 600e3, 10e3, 15.0
    xi = lgl_nodes()
    fmin = (xi[1] + 1.0) / 2.0
    dt = C * fmin * (Lz / nez) / C_S
    g = pkg.Numa(nex, nex, nez, L, L, Lz, n, dt)
    lev = g.reference_levels()
    h = L / nex
    ax = np.concatenate([e * h + (1.0 + xi[:-1]) * h / 2.0 for e in range(nex)] + [[L]])

    def state(seed, **kw):
        return torch.from_numpy(synthetic.random_state(ax, ax, lev["z"], L, L, Lz, lev["rho0"],
                                                       lev["theta0"], seed, **kw)).cuda()
    q0 = state(5001, vel=5.0)
    target = state(5002)[4].contiguous()
    dq, lam = state(5003, vel=3.0), state(5004, vel=2.0)

    def misfit(q):
        qT = g.trajectory(q, nsteps, every)
        return 0.5 * ((qT[4] - target) ** 2).sum()

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
    fwd = bwd = tlm = 0.0
    for r in range(warmup + reps):
        x = q0.clone().requires_grad_(True)
        torch.cuda.synchronize()
        ev[0].record()
        J = misfit(x)
        ev[1].record()
        J.backward()
        ev[2].record()
        ev[2].synchronize()
        if r >= warmup:
            fwd += ev[0].elapsed_time(ev[1]) / reps
            bwd += ev[1].elapsed_time(ev[2]) / reps
    grad = x.grad
    for r in range(warmup + reps):
        torch.cuda.synchronize()
        ev[0].record()
        _, dqT = g.step_imex1d_tlm(q0, dq, nsteps)
        ev[1].record()
        ev[1].synchronize()
        if r >= warmup:
            tlm += ev[0].elapsed_time(ev[1]) / reps
    # per-kernel times of one adjoint sweep
    qT, ckpt = g.forward_checkpointed(q0, nsteps, every)
    g.profile(True)
    lam0 = g.adjoint_checkpointed(ckpt, nsteps, every, lam)
    kern = {}
    for name, kind in (("k_rhs_adj (weights + gather)", pkg.K_RHS_ADJ),
                       ("k_stage_adj", pkg.K_STAGE_ADJ), ("k_rhs (recompute)", pkg.K_RHS),
                       ("k_stage (recompute)", pkg.K_STAGE)):
        t, cnt = g.profile_read(kind)
        kern[name] = {"launches": cnt, "ms_per_launch": round(t / max(cnt, 1), 5)}
    g.profile(False)
    # checks: dot product of the run, centred differences of J
    a = float((lam * dqT).sum())
    b = float((lam0 * dq).sum())
    eps = 1e-6
    d = state(5005, vel=3.0)
    with torch.no_grad():
        fd = (float(misfit(q0 + eps * d)) - float(misfit(q0 - eps * d))) / (2 * eps)
    ad = float((grad * d).sum())
    sim = nsteps * dt
    nodes = g.nnode
    g.close()
    return {"workload": "16x16x8 hex elements over 600x600x10 km, N=4 (65x65 columns x 33 levels), "
                        "%d HEVI 1D-IMEX ARK2 steps at C=15, checkpoints every %d" % (nsteps, every),
            "nodes": int(nodes), "dt_s": round(dt, 4),
            "forward_checkpointed_ms": round(fwd, 3), "adjoint_ms": round(bwd, 3),
            "gradient_ms": round(fwd + bwd, 3), "adjoint_over_forward": round(bwd / fwd, 3),
            "tlm_run_ms": round(tlm, 3),
            "gradients_per_s": round(1e3 / (fwd + bwd), 2),
            "sim_s_per_wall_s_of_gradient": round(sim / ((fwd + bwd) / 1e3), 1),
            "kernels": kern,
            "dot_product_rel_diff": float("%.3g" % (abs(a - b) / abs(a))),
            "fd_rel_diff_step_1e-6": float("%.3g" % (abs(fd - ad) / abs(ad))),
            "finite": bool(torch.isfinite(grad).all().item())}


ORACLE_HALO = 3        # elements of halo per block: one ARK2 step evaluates R three times


def oracle_procs():
    """Worker processes for the oracle timings: one single-threaded process per host core
    (NUMA_ORACLE_PROCS overrides)."""
    v = os.environ.get("NUMA_ORACLE_PROCS")
    return max(1, int(v)) if v else (os.cpu_count() or 1)


def oracle_blocks(nex, ney, nproc):
    """Split an nex x ney element grid into nproc rectangular blocks, px x py = nproc with
    px, py as close as possible: list of (ex0, ex1, ey0, ey1)."""
    px = max(d for d in range(1, int(nproc ** 0.5) + 1) if nproc % d == 0)
    py = nproc // px
    if px > nex or py > ney:
        raise ValueError("more blocks than elements")
    cx = [nex * i // px for i in range(px + 1)]
    cy = [ney * j // py for j in range(py + 1)]
    return [(cx[i], cx[i + 1], cy[j], cy[j + 1]) for j in range(py) for i in range(px)]


def _oracle_block_worker(mesh, dt, block, qpath, opath, warmup, steps, barrier, results):
    """One process of the partitioned oracle run: its block of elements plus a halo of
    ORACLE_HALO elements (clipped at the real walls) as a box of its own, ARK2 steps of
    that window from the same input, the owned nodes of the last result written out.
    The halo makes the owned nodes exact: a window's artificial walls corrupt one more
    element ring per evaluation of R, three per step."""
    import numpy as np
    from oracle import ark2
    from oracle.column import Column
    from oracle.mesh import BoxMesh
    nex, ney, nez, Nn, Lx, Ly, Lz = mesh
    ex0, ex1, ey0, ey1 = block
    wx0, wx1 = max(0, ex0 - ORACLE_HALO), min(nex, ex1 + ORACLE_HALO)
    wy0, wy1 = max(0, ey0 - ORACLE_HALO), min(ney, ey1 + ORACLE_HALO)
    dx, dy = Lx / nex, Ly / ney
    m = BoxMesh(wx1 - wx0, wy1 - wy0, nez, Nn, (wx1 - wx0) * dx, (wy1 - wy0) * dy, Lz)
    H = ark2.HEVI(m, Column(m), dt)
    nxg, nyg, M = nex * Nn + 1, ney * Nn + 1, nez * Nn + 1
    q0 = np.load(qpath, mmap_mode="r").reshape(5, nyg, nxg, M)
    q = np.ascontiguousarray(q0[:, wy0 * Nn:wy1 * Nn + 1, wx0 * Nn:wx1 * Nn + 1, :]).reshape(5, -1)
    del q0
    for _ in range(warmup):
        H.step(q, 1)
    barrier.wait()
    for _ in range(steps):
        out = H.step(q, 1)
    barrier.wait()
    # owned node columns: [e0 N, e1 N), plus the last node at the east / north wall
    ox1 = ex1 * Nn + (1 if ex1 == nex else 0)
    oy1 = ey1 * Nn + (1 if ey1 == ney else 0)
    o = np.load(opath, mmap_mode="r+").reshape(5, nyg, nxg, M)
    w = out.reshape(5, m.nyg, m.nxg, M)
    o[:, ey0 * Nn:oy1, ex0 * Nn:ox1, :] = w[:, (ey0 - wy0) * Nn:oy1 - wy0 * Nn,
                                             (ex0 - wx0) * Nn:ox1 - wx0 * Nn, :]
    o.flush()
    results.put(m.ncol)


def oracle_partitioned(mesh, dt, q0, nproc, warmup, steps, timeout=3600):
    """The oracle, as it stands, over a whole mesh on nproc single-threaded processes (spawned
    fresh, so no GPU state is inherited).  Each process advances its block of columns (plus
    a halo) by `steps` ARK2 steps from the same input q0 after `warmup` untimed ones; the
    parent times from the barrier that starts the timed steps to the one that ends them, so
    the figure is the slowest process's.  Returns (seconds per step, the assembled result
    of one step, columns computed per step including the halos)."""
    import multiprocessing as mp
    import tempfile
    nex, ney = mesh[0], mesh[1]
    blocks = oracle_blocks(nex, ney, nproc)
    tmp = "/dev/shm" if os.path.isdir("/dev/shm") and os.access("/dev/shm", os.W_OK) else None
    with tempfile.TemporaryDirectory(dir=tmp) as d:
        qpath, opath = os.path.join(d, "q0.npy"), os.path.join(d, "out.npy")
        np.save(qpath, np.ascontiguousarray(q0, dtype=np.float64))
        np.lib.format.open_memmap(opath, mode="w+", dtype=np.float64, shape=q0.shape).flush()
        saved = {v: os.environ.get(v) for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS",
                                                  "MKL_NUM_THREADS")}
        for v in saved:
            os.environ[v] = "1"
        ctx = mp.get_context("spawn")
        barrier = ctx.Barrier(len(blocks) + 1, timeout=timeout)
        results = ctx.Queue()
        procs = [ctx.Process(target=_oracle_block_worker,
                             args=(mesh, dt, b, qpath, opath, warmup, steps, barrier, results))
                 for b in blocks]
        try:
            for pr in procs:
                pr.start()
            barrier.wait()
            t0 = time.perf_counter()
            barrier.wait()
            t1 = time.perf_counter()
            cols = sum(results.get(timeout=timeout) for _ in procs)
            for pr in procs:
                pr.join(timeout)
        finally:
            for pr in procs:
                if pr.is_alive():
                    pr.kill()
            for v, x in saved.items():
                if x is None:
                    os.environ.pop(v, None)
                else:
                    os.environ[v] = x
        if any(pr.exitcode != 0 for pr in procs):
            raise RuntimeError("an oracle worker failed")
        out = np.array(np.load(opath))
    return (t1 - t0) / max(steps, 1), out, cols


def workload_state():
    """The benchmark's input on the host: the seeded balanced state of the workload."""
    import synthetic
    from oracle.column import Column
    from oracle.mesh import BoxMesh
    m = BoxMesh(NEX, NEY, NEZ, N, LX, LY, LZ)
    col = Column(m)
    xg, yg, zg = m.coords()
    return synthetic.balanced_state(xg, yg, zg, LX, LY, LZ, col.rho0, col.theta0, SEED)


def oracle_workload(warmup, steps, nproc):
    """The partitioned oracle on the whole benchmark workload: (s per step, procs, sample)."""
    sec, _, cols = oracle_partitioned((NEX, NEY, NEZ, N, LX, LY, LZ), dt_for(C_MAIN),
                                      workload_state(), nproc, warmup, steps)
    full_cols = (NEX * N + 1) * (NEY * N + 1)
    bl = oracle_blocks(NEX, NEY, nproc)
    sample = ("the whole %dx%dx%d-element mesh (%d columns) every step: %d single-threaded "
              "processes, each on a block of about %dx%d elements with a %d-element halo "
              "(%.2fx the columns), %d timed ARK2 steps at C=15 from the same input after %d "
              "untimed; time from the barrier that starts them to the one that ends them"
              % (NEX, NEY, NEZ, full_cols, nproc, bl[0][1] - bl[0][0], bl[0][3] - bl[0][2],
                 ORACLE_HALO, cols / full_cols, steps, warmup))
    return sec, nproc, sample


def cpu_baseline(seconds):
    """The oracle, as it stands, on every host core over the whole workload: one timed ARK2
    step of the full mesh after one untimed step (oracle_partitioned).  `seconds` is
    unused: the sample is the whole mesh once."""
    nproc = oracle_procs()
    try:
        sec, nproc, sample = oracle_workload(1, 1, nproc)
    except Exception as e:
        return {"value": None, "unit": "sim-s/wall-s", "cores": nproc, "kind": "oracle",
                "sample": "failed: " + str(e)[:200]}
    return {"value": dt_for(C_MAIN) / sec, "unit": "sim-s/wall-s", "cores": nproc,
            "kind": "oracle", "ms_per_step": round(sec * 1e3, 1), "sample": sample}


def run_reference(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if world > 1 and rank != 0:
        return
    nproc = oracle_procs()
    sec, nproc, sample = oracle_workload(args.warmup, args.steps, nproc)
    dt = dt_for(C_MAIN)
    ms_step = sec * 1e3
    value = dt / sec
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "sim-s/wall-s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": {"workload": WORKLOAD, "C_V": C_MAIN},
        "cpu_baseline": {"value": value, "unit": "sim-s/wall-s", "cores": nproc, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "sim-s/wall-s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the precision-form workload")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)      # at least three untimed warm-up steps
    if args.impl == "reference":
        run_reference(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
