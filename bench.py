#!/usr/bin/env python
"""Benchmark of the GPU splitting conic solver on the large mixed-cone program.

Workload (default): n = 1e6 variables, m = 2e6 rows, nnz(A) = 2e7 with
power-law row lengths, cones zero 1e5 / SOC 2e4 blocks of 3..50 / exp 1e4 /
nonnegative rest, built by the Sec. 6.6 generator (seed 0).  A step is one
ADMM iteration of Eq. "e-SCS" (subspace projection by warm-started PCG,
cone projection, dual update) on that problem; the metric is ADMM
iterations per second with A resident in HBM, FP32 sparse products and CG,
FP64 iterates and checks.  The JSON line also carries the time to the 1e-4
tolerances, the end-to-end rate through the C ABI with host buffers, the
roofline of the dominant kernel, the CPU oracle's rate and the SM clocks.

``--impl reference`` times the FP64 CPU oracle (the paper's indirect method
restated in numpy/scipy) on the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "ADMM iters/s and time-to-1e-4 (s); SpMV/CG HBM GB/s vs peak; warm/batched vs plain"
FALLBACK_HBM_GBS = 6800.0


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["mixed", "mixed_small", "sdp", "sdp_small", "sdp_blocks", "lp",
                                           "portfolio_batch", "portfolio_batch_small", "lasso_warm",
                                           "lasso_warm_small", "mlp_train"] + sorted(PAPER_APPS),
                    default="mixed")
    ap.add_argument("--train", type=int, default=None, help="training members of a lasso_warm workload")
    ap.add_argument("--epochs", type=int, default=30)
    ap.add_argument("--plain-sample", type=int, default=64,
                    help="programs of a batched workload solved one by one by the plain solver")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-solve", action="store_true", help="skip the time-to-1e-4 solve")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=20.0)
    ap.add_argument("--solve-seconds", type=float, default=90.0, help="time limit of the time-to-1e-4 leg")
    ap.add_argument("--solve-iters", type=int, default=100000, help="iteration limit of the time-to-1e-4 leg")
    ap.add_argument("--linsys", type=int, default=0, choices=[0, 1],
                    help="subspace step: 0 indirect (PCG), 1 direct (cached dense (I + A^T A)^-1, n <= 8192)")
    return ap.parse_args()


def reduce_scalar(x, op, device="cuda"):
    """x reduced over the ranks of the default process group ("max" or
    "sum"); x itself when there is no group.  device: where the backend
    exchanges tensors ("cuda" for NCCL, "cpu" for gloo)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


def replica_rate(units_local, seconds_local, device="cuda"):
    """Whole-job rate of independent replicas: the units every rank did,
    divided by the slowest rank's time (the timed region ends when the last
    replica ends).  Returns (rate, units_total, seconds_max)."""
    units = reduce_scalar(units_local, "sum", device)
    secs = reduce_scalar(seconds_local, "max", device)
    return units / secs, units, secs


def dist_env():
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


# The paper's application workloads at the sizes of its Tables 1-4 (small and
# medium), built as the paper prints them (Sec. 6.2-6.5), with the paper's
# own GPU result for context: the indirect method on a GeForce GTX Titan X,
# eps 1e-3, setup included (its standard forms differ from the printed
# SOCP/SDP for the lasso, portfolio and RPCA tables: see n, m, nnz).
PAPER_APPS = {
    "paper_lasso": (("lasso_paper", dict(p=10_000, q=2_000)), "lasso (Sec. 6.2) small: p=1e4 features, q=2e3 "
                    "measurements, dense F", dict(gpu_s=4.6, iters=400, n=2001, m=22002, nnz=3.8e6)),
    "paper_lasso_medium": (("lasso_paper", dict(p=30_000, q=6_000)), "lasso (Sec. 6.2) medium: p=3e4, q=6e3, "
                           "dense F", dict(gpu_s=22.0, iters=540, n=6001, m=66002, nnz=3.4e7)),
    "paper_portfolio": (("portfolio_paper", dict(p=100_000, q=100)), "portfolio (Sec. 6.3, both risk SOCs) small: "
                        "p=1e5 assets, q=100 factors", dict(gpu_s=27.8, iters=500, n=100103, m=200104, nnz=1.3e6)),
    "paper_portfolio_medium": (("portfolio_paper", dict(p=500_000, q=500)), "portfolio (Sec. 6.3) medium: p=5e5, "
                               "q=500", dict(gpu_s=184.0, iters=440, n=500503, m=1000504, nnz=2.5e7)),
    "paper_rpca": (("rpca_paper", dict(p=100)), "robust PCA (Sec. 6.4) small: p=q=100, rank 10, PSD block of "
                   "order 200", dict(gpu_s=6.1, iters=120, n=10001, m=40101, nnz=5.0e4)),
    "paper_logreg": (("logreg_paper", dict(p=100, q=10_000)), "l1 logistic regression (Sec. 6.5) small: p=100, "
                     "q=1e4 samples, 2e4 exponential cones", dict(gpu_s=4.4, iters=280, n=30200, m=70200, nnz=1.6e5)),
    "paper_logreg_medium": (("logreg_paper", dict(p=1_000, q=100_000)), "l1 logistic regression (Sec. 6.5) medium: "
                            "p=1e3, q=1e5", dict(gpu_s=120.0, iters=380, n=302000, m=702000, nnz=1.0e7)),
}


def make_problem(workload, seed):
    from paper_1312_3039_gb300 import synth
    if workload in PAPER_APPS:
        (fn, kw), desc, _paper = PAPER_APPS[workload]
        P = getattr(synth, fn)(seed, **kw)
        return P, f"{desc} (n={P.n}, m={P.m}, nnz={P.A.nnz})"
    if workload == "mixed":
        return synth.mixed(seed), ("mixed-cone program n=1e6 m=2e6 nnz=2e7 (power-law rows; zero 1e5, "
                                   "SOC 2e4 blocks of 3-50, exp 1e4, nonneg rest)")
    if workload == "mixed_small":
        return synth.mixed_small(seed, scale=50), "mixed-cone program n=2e4 m=4e4 nnz=4e5 (same recipe)"
    if workload == "sdp":
        return synth.sdp(seed), ("SDP-heavy program n=2e5 m=578384 nnz=1.16e8 (64 PSD blocks of order 128 in svec "
                                 "form, 5e4 nonneg; uniform A at density 1e-3; 8 blocks with eigenvalues over "
                                 "1e-7..1)")
    if workload == "sdp_blocks":
        return (synth.sdp(seed, n=20000, density=1e-4),
                "PSD blocks of the SDP-heavy program with a small A: 64 PSD blocks of order 128 + 5e4 nonneg, "
                "n=2e4, density 1e-4 (nnz 1.16e6)")
    if workload == "sdp_small":
        return (synth.sdp(seed, n=4000, n_psd=16, order=64, n_nonneg=2000, density=2e-3, n_ill=2),
                "SDP program n=4e3 m=35280 (16 PSD blocks of order 64, 2e3 nonneg; density 2e-3; 2 ill blocks)")
    return synth.lp(seed), "sparse LP n=200 m=400 (zero 100, nonneg 300), 5% density"


def measured_hbm_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        time.sleep(0.3)

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[5:9]):
                    if val.lower().startswith("active"):
                        reasons.add(name)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def spmv_bytes(P, it, cg, elt=4):
    """Algorithmic bytes of the SpMV launches (kind 0: with A, kind 1: with
    A^T) over ``it`` ADMM iterations with ``cg`` CG steps in total.  Each
    launch streams its CSR arrays once (elt-byte values, 4-byte column
    indices and row pointers), gathers its input vector once from L2 (counted
    once: elt bytes per entry) and moves its epilogue's vectors."""
    m, n, nnz = P.m, P.n, P.A.nnz
    mat_a = (elt + 4) * nnz + 4 * (m + 1)
    mat_at = (elt + 4) * nnz + 4 * (n + 1)
    k3 = mat_a + elt * n + elt * m                                # p gathered; q written
    k2 = mat_at + elt * m + (8 + 8 + elt + elt) * n + 2 * elt * n  # y_acc gathered; u_x, c, z, diag read; r, p written
    k4 = (mat_at + elt * m + 4 * elt * n + 2 * elt * n            # q gathered; p, z, r, diag read; z, r written
          + 5 * elt * m)                                          # side task: q, y_acc, az read; y_acc, az written
    # kind 0 counts the CG products q = A p only (the profiled pass does not
    # time K1, whose product runs on one iteration in 20)
    return {0: cg * k3, 1: it * k2 + cg * k4, "per_launch": {"A_cg": k3, "At_cg": k4}}


def psd_flops(orders, sweeps_per_block):
    """Flop model of one PSD launch (every block once), FP32 arithmetic:
    re-orthonormalisation of V and the similarity V^T X V (4 products of
    order ne: 8 ne^3), the Jacobi sweeps and the reconstruction over half of
    the eigenvalues (ne^3).  Orders up to 48 (ne = n rounded up to 4): a
    sweep is ne - 1 rounds of 12 h^2 + 6 n h flops (h = ne / 2: both sides of
    the lower 2 x 2 blocks and the rows of V).  Above (ne = n rounded up to
    16, nb = ne / 8 blocks, P = ne / 16 block pairs): a sweep is nb - 1
    block rounds, each with the rotations of every block pair's 16 x 16
    subproblem (15 rounds in the first block round of a sweep, 8 in the
    others; a round is 36 2 x 2 blocks of 24 flops and 16 x 8 Q updates of 6
    flops), the P (P - 1) / 2 off-diagonal blocks Q_k^T X_kl Q_l (two
    16 x 16 x 16 products each) and V[:, R] <- V[:, R] Q (32 n ne flops over
    all pairs), counted as the kernel performs them."""
    tot = 0.0
    for n in orders:
        if n <= 48:
            ne = max(4, (n + 3) // 4 * 4)
            h = ne // 2
            sweep = (ne - 1) * (12.0 * h * h + 6.0 * n * h)
        else:
            ne = (n + 15) // 16 * 16
            nb, npairs = ne // 8, ne // 16
            rnd = 36 * 24.0 + 16 * 8 * 6.0
            sub = npairs * rnd * (15 + 8 * (nb - 2))
            sweep = sub + (nb - 1) * (npairs * (npairs - 1) / 2 * 4.0 * 16 ** 3 + 32.0 * n * ne)
        tot += 8.0 * ne ** 3 + sweeps_per_block * sweep + 1.0 * ne ** 3
    return tot


def fp32_alu_peak_tflops(sm_mhz):
    """FP32 FMA peak from the unit counts: 152 SMs x 128 FP32 lanes x 2 flops
    per clock at the sampled SM clock (max 2070 MHz)."""
    return 152 * 128 * 2 * (sm_mhz or 2070.0) * 1e6 / 1e12


def cpu_oracle_job(workload, seed, seconds, queue):
    """CPU baseline (runs in a spawned process, in parallel with the GPU
    legs): the FP64 oracle's indirect method on the same problem, one
    thread; ADMM iterations are timed after its setup for about `seconds`."""
    try:
        P, _ = make_problem(workload, seed)
        from oracle import admm
        t0 = time.perf_counter()
        S = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings(linsys="indirect"))
        setup = time.perf_counter() - t0
        t1 = time.perf_counter()
        it = 0
        while True:
            S.step()
            it += 1
            if time.perf_counter() - t1 >= seconds:
                break
        queue.put({"iters": it, "seconds": time.perf_counter() - t1, "setup": setup})
    except Exception as e:  # report, never hang the benchmark
        queue.put({"error": repr(e)})


ORACLE_ERR_SCALES = (500, 50)


def oracle_err_job(seed, queue):
    """FP64 oracle solves of the down-scaled siblings of the large mixed
    program (the same generator divided by 500 and by 50), with the GPU
    engine's method and settings (indirect CG, (1/k)^1.5 capped at 0.3 x the
    last step, 50 CG steps at most, eps 1e-4); runs in a spawned process
    alongside the GPU legs.  The full-size program is beyond the oracle."""
    try:
        from oracle import admm
        from paper_1312_3039_gb300 import synth
        out = {}
        for sc in ORACLE_ERR_SCALES:
            P = synth.mixed_small(seed, scale=sc)
            t0 = time.perf_counter()
            r = admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(linsys="indirect", cg_max_iters=50))
            out[sc] = {"status": r.status, "iters": r.iters, "pobj": r.pobj, "x": r.x, "y": r.y, "s": r.s,
                       "seconds": time.perf_counter() - t0}
        queue.put(out)
    except Exception as e:
        queue.put({"error": repr(e)})


def two_point_bound(P, x1, y1, s1, x2, y2, s2):
    """Largest objective difference weak duality allows between two points
    with these residuals (s in K, y in K*): c^T x1 - c^T x2 lies in
    [-g2 - ||y2|| ||r_p1|| - ||x1|| ||r_d2||, g1 + ||y1|| ||r_p2|| + ||x2|| ||r_d1||],
    r_p = A x + s - b, r_d = A^T y + c, g = c^T x + b^T y."""
    import numpy as np

    def parts(x, y, s):
        return (float(np.linalg.norm(P.A @ x + s - P.b)), float(np.linalg.norm(P.A.T @ y + P.c)),
                float(P.c @ x + P.b @ y), float(np.linalg.norm(x)), float(np.linalg.norm(y)))
    rp1, rd1, g1, nx1, ny1 = parts(x1, y1, s1)
    rp2, rd2, g2, nx2, ny2 = parts(x2, y2, s2)
    return max(g2 + ny2 * rp1 + nx1 * rd2, g1 + ny1 * rp2 + nx2 * rd1)


def oracle_err(seed, orc, common):
    """Each precision's result on the siblings stated against the FP64
    oracle: objective error (relative to 1 + |oracle objective|), the
    two-point weak-duality bound on it, residuals, iterations."""
    from paper_1312_3039_gb300 import scs, synth
    if orc is None or "error" in orc:
        return {"error": None if orc is None else orc["error"]}
    res = {}
    for sc in ORACLE_ERR_SCALES:
        P = synth.mixed_small(seed, scale=sc)
        o = orc[sc]
        row = {"oracle": {"status": o["status"], "iters": o["iters"], "pobj": o["pobj"],
                          "seconds": o["seconds"]}, "p_star": P.p_star}
        for prec in (1, 0):
            kw = dict(common)
            kw["precision"] = prec
            st, x, y, s, info = scs.solve(P.A, P.b, P.c, P.cone, **kw)
            row["fp32" if prec else "fp64"] = {
                "status": int(st), "iters": info["iters"], "pobj": info["pobj"],
                "rel_err_vs_oracle": abs(info["pobj"] - o["pobj"]) / (1 + abs(o["pobj"])),
                "two_point_bound_rel": two_point_bound(P, x, y, s, o["x"], o["y"], o["s"]) / (1 + abs(o["pobj"])),
                "rel_err_vs_p_star": abs(info["pobj"] - P.p_star) / (1 + abs(P.p_star)),
                "res_pri": info["res_pri"], "res_dual": info["res_dual"], "gap": info["gap"]}
        res["mixed_div%d" % sc] = row
    return res


def spmv_device_digest():
    """Digest of the device code behind the SpMV traffic record: the SpMV
    kernels (csrc/spmv.cuh up to its host-side layout builder), the CG
    epilogues of the two measured launches (EpiACG, EpiAtCG in
    csrc/kernels.cuh) and csrc/common.cuh's device helpers.  Host code (the
    layout builder, the engine) is left out, so host-only changes keep it."""
    import hashlib
    import re
    src = os.path.join(ROOT, "paper_1312_3039_gb300", "csrc")
    with open(os.path.join(src, "spmv.cuh")) as f:
        spmv = f.read()
    cut = spmv.find("// Stored layout of one CSR matrix")
    parts = [spmv[:cut if cut >= 0 else len(spmv)]]
    with open(os.path.join(src, "kernels.cuh")) as f:
        ker = f.read()
    for name in ("EpiACG", "EpiAtCG"):
        m = re.search(r"struct %s \{.*?\n\};" % name, ker, re.S)
        parts.append(m.group(0) if m else "")
    with open(os.path.join(src, "common.cuh")) as f:
        parts.append(f.read())
    h = hashlib.sha256()
    for t in parts:
        h.update(t.encode())
    return h.hexdigest()[:16]


def traffic_record(kind):
    """DRAM bytes per launch of SpMV kind 0 (A) / 1 (A^T) from the committed
    ncu summary, if the kernels' device code is unchanged since that capture."""
    digest = spmv_device_digest()
    path = os.path.join(ROOT, "profiles", "spmv_traffic.txt")
    try:
        with open(path) as f:
            for line in f:
                parts = line.split()
                if len(parts) == 4 and parts[0] == "traffic" and int(parts[1]) == kind and parts[3] == digest:
                    return float(parts[2]), digest
    except OSError:
        pass
    return None, digest


def run_reference(args):
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    if args.workload.startswith("portfolio_batch"):
        return run_reference_batch(args)
    P, desc = make_problem(args.workload, args.seed)
    from oracle import admm
    t0 = time.perf_counter()
    S = admm.HSDSolver(P.A, P.b, P.c, P.cone, admm.Settings(linsys="indirect"))
    setup = time.perf_counter() - t0
    for _ in range(args.warmup):
        S.step()
    t1 = time.perf_counter()
    for _ in range(args.steps):
        S.step()
    el = time.perf_counter() - t1
    value = args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (Sec. 6.6 generator, seed %d)" % args.seed,
        "config": {"workload": desc, "precision": "fp64", "linsys": "indirect CG (oracle)"},
        "cpu_baseline": {"value": value, "unit": "iter/s", "cores": 1, "kind": "oracle",
                         "sample": f"{args.steps} ADMM iterations after {args.warmup} warm-up "
                                   f"(setup {setup:.1f} s not timed)"},
        "e2e": {"value": value, "unit": "iter/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_batch(args):
    """Reference arm of a batched workload: the FP64 oracle solving the
    programs of a stratified sample one by one (one thread)."""
    import multiprocessing as mp
    q = mp.get_context("spawn").Queue()
    per_step = max(args.cpu_seconds / max(args.steps, 1), 1.0)
    t0 = time.perf_counter()
    got = []
    for _ in range(args.steps):
        cpu_batch_job(args.workload, args.seed, per_step, q)
        got.append(q.get())
    el = time.perf_counter() - t0
    done = sum(r.get("programs", 0) for r in got)
    _, desc = batch_programs(args.workload, args.seed)
    value = done / el if el > 0 else None
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "programs/s", "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / max(args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (Sec. 6.3 portfolio form, seed %d)" % args.seed,
            "config": {"workload": desc, "precision": "fp64", "linsys": "direct (oracle)"},
            "cpu_baseline": {"value": value, "unit": "programs/s", "cores": 1, "kind": "oracle",
                             "sample": f"{done} programs of a stratified sample, one thread"},
            "e2e": {"value": value, "unit": "programs/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_gb300(args):
    world, rank, local = dist_env()
    cpu_proc = cpu_q = None
    if rank == 0 and not args.no_cpu_baseline:
        # spawned before any CUDA call, so the child never inherits a context
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        cpu_q = ctx.Queue()
        cpu_proc = ctx.Process(target=cpu_oracle_job, args=(args.workload, args.seed, args.cpu_seconds, cpu_q),
                               daemon=True)
        cpu_proc.start()
    err_proc = err_q = None
    if rank == 0 and not args.no_cpu_baseline and args.workload == "mixed":
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        err_q = ctx.Queue()
        err_proc = ctx.Process(target=oracle_err_job, args=(args.seed, err_q), daemon=True)
        err_proc.start()
    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1312_3039_gb300 import scs

    P, desc = make_problem(args.workload, args.seed)
    # a stream of our own (the default stream's handle is 0, which the library
    # would replace by a private stream that torch's events do not see)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # the small LP runs in FP64 throughout (its parity configuration); the
    # other programs in the mixed-precision engine
    prec = 0 if args.workload == "lp" else 1
    common = dict(precision=prec, device=local, cuda_stream=stream.cuda_stream, linsys=args.linsys)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        return reduce_scalar(x, "max")

    def sum_over_ranks(x):
        return reduce_scalar(x, "sum")

    S = scs.Solver(P.A, P.b, P.c, P.cone, time_limit_s=args.solve_seconds, max_iters=args.solve_iters, **common)
    # warm-up iterations, then exactly `steps` timed iterations
    S.iterate(args.warmup)
    torch.cuda.synchronize()
    barrier()
    it0, cg0 = S.counters()
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    barrier()
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")      # ncu --nvtx-include "timed/" selects these launches
    e0.record(stream)
    # the solve's work per iteration: the Sec. 3.5 tests every 20 iterations
    # (two FP64 products on the device and a host read of the status word)
    S.iterate_checked(args.steps)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    it1, cg1 = S.counters()
    value, iters_done, secs = replica_rate(it1 - it0, e0.elapsed_time(e1) / 1e3)
    ms = secs * 1e3
    cg_steps = cg1 - cg0
    # per iteration K1 (product or return), K1', K2, K6, K7 (+ KP with PSD
    # blocks) and K3, K4, K5 per CG step; two check products per 20 iterations
    ci = int(S.settings.check_interval) or 1
    launches = (6 if getattr(P.cone, "s", ()) else 5) * (it1 - it0) + 3 * cg_steps + 2 * (-(-args.steps // ci))

    # roofline of the dominant kernel (CUDA events around each SpMV launch)
    has_psd = bool(getattr(P.cone, "s", ()))
    psd0 = S.psd_counters() if has_psd else None
    # launched one by one (not through the graph: ncu does not profile kernel
    # nodes of graphs with conditional nodes): ncu --nvtx-include "profiled/"
    torch.cuda.nvtx.range_push("profiled")
    S.iterate_profiled(5)
    torch.cuda.nvtx.range_pop()
    prof = {k: S.kernel_time(k) for k in (0, 1, 2, 3, 4)}
    it_p, cg_p = S.counters()
    # counters include the profiled iterations: take CG steps of those 5 from
    # the launch counts (kind 0 = the CG launches of q = A p)
    cg_prof = prof[0][1]
    byt = spmv_bytes(P, 5, cg_prof, elt=8 if prec == 0 else 4)
    kind = 0 if prof[0][0] >= prof[1][0] else 1
    achieved = byt[kind] / (prof[kind][0] / 1e3) / 1e9
    peak, peak_src = measured_hbm_peak()
    names = {0: "spmv_A (q = A p, y_acc init)", 1: "spmv_At (A^T q + CG update)"}
    traffic, src_digest = traffic_record(kind)
    roofline = {"bound": "hbm", "kernel": names[kind], "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "peak_source": peak_src, "traffic": traffic,
                "kernel_src_digest": src_digest,
                "algorithmic_bytes_per_cg_launch": byt["per_launch"]["A_cg" if kind == 0 else "At_cg"],
                "avg_launch_us": 1e3 * prof[kind][0] / prof[kind][1],
                "other_kernel_avg_us": 1e3 * prof[1 - kind][0] / max(prof[1 - kind][1], 1),
                "projection_avg_us": 1e3 * prof[2][0] / max(prof[2][1], 1),
                "psd_projection_avg_us": 1e3 * prof[3][0] / prof[3][1] if prof[3][1] else None,
                "direct_step_avg_us": 1e3 * prof[4][0] / prof[4][1] if prof[4][1] else None}

    psd = None
    if has_psd and prof[3][1]:
        calls, sweeps, fp64 = (b - a for a, b in zip(psd0, S.psd_counters()))
        per_block = sweeps / max(calls, 1)
        avg_us = 1e3 * prof[3][0] / prof[3][1]
        flops = psd_flops(P.cone.s, per_block)
        peak_t = fp32_alu_peak_tflops(clk.get("sm_mhz"))
        achieved_t = flops / (avg_us * 1e-6) / 1e12
        psd = {"bound": "alu", "kernel": "psd_project_kernel (Jacobi per block, blocked above order 48; one CTA per block)",
               "achieved": achieved_t, "peak": peak_t, "unit": "TFLOP/s", "frac": achieved_t / peak_t,
               "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 flop x sampled SM clock",
               "avg_launch_us": avg_us, "blocks": len(P.cone.s), "sweeps_per_block": per_block,
               "fp64_reconstructed_frac": fp64 / max(calls, 1), "flops_per_launch": flops}

    # time to the 1e-4 tolerances from a cold start, data resident
    solve = None
    if not args.no_solve:
        psd_s0 = S.psd_counters() if has_psd else None
        st, x, y, s, info = S.solve()
        if psd is not None:
            c_, sw_, f_ = (b - a for a, b in zip(psd_s0, S.psd_counters()))
            psd["solve_sweeps_per_block"] = sw_ / max(c_, 1)
            psd["solve_fp64_reconstructed_frac"] = f_ / max(c_, 1)
        solve = {"status": int(st), "iters": info["iters"], "seconds": info["solve_s"],
                 "avg_cg_per_iter": info["cg_iters"] / max(info["iters"], 1),
                 "pobj": info["pobj"], "p_star": P.p_star,
                 "rel_err_vs_p_star": abs(info["pobj"] - P.p_star) / (1 + abs(P.p_star)) if P.p_star else None,
                 "setup_s": info["setup_s"]}
    S.close()

    # end to end through the C ABI with host buffers: scs_init from the host
    # CSC, `steps` iterations of scs_solve (tolerances 0), outputs to host
    e2e = None
    if not args.no_e2e:
        torch.cuda.synchronize()
        barrier()
        t0 = time.perf_counter()
        S2 = scs.Solver(P.A, P.b, P.c, P.cone, max_iters=args.steps, eps_pri=0.0, eps_dual=0.0, eps_gap=0.0,
                        eps_infeas=0.0, eps_unbdd=0.0, **common)
        t1 = time.perf_counter()
        st, x, y, s, info = S2.solve()
        t2 = time.perf_counter()
        S2_setup = info.get("setup_s")
        S2.close()
        torch.cuda.synchronize()
        t3 = time.perf_counter()
        el = max_over_ranks(t3 - t0)
        h2d = 8 * (P.n + 1) + 12 * P.A.nnz + 8 * P.m + 8 * P.n
        d2h = 8 * (P.n + 2 * P.m)
        e2e = {"value": sum_over_ranks(args.steps) / el, "unit": "iter/s",
               "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
               "seconds": el, "includes": "scs_init (host CSC->CSR, H2D, equilibration, M^-1 h) + scs_solve "
                                          f"({args.steps} iterations) + D2H of x, y, s",
               "breakdown_s": {"scs_init": t1 - t0, "scs_solve": t2 - t1, "scs_finish": t3 - t2,
                               "engine_setup": S2_setup}}

    cpu = None
    if cpu_proc is not None:
        try:
            r = cpu_q.get(timeout=600)
        except Exception as e:
            r = {"error": "no result: " + repr(e)}
        cpu_proc.join(timeout=10)
        if "error" in r:
            cpu = {"value": None, "unit": "iter/s", "cores": 1, "kind": "oracle", "sample": r["error"]}
        else:
            cpu = {"value": r["iters"] / r["seconds"], "unit": "iter/s", "cores": 1, "kind": "oracle",
                   "sample": f"{r['iters']} ADMM iterations ({r['seconds']:.1f} s) of the FP64 oracle (indirect "
                             f"CG, scipy sparse, one thread) on the same problem after its setup "
                             f"({r['setup']:.1f} s, not timed); run in a separate process alongside the GPU legs"}

    # the paper's own setting for its application tables: eps 1e-3, time from
    # the host data (scs_init included), one cold solve
    paper_ctx = None
    if args.workload in PAPER_APPS:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S3 = scs.Solver(P.A, P.b, P.c, P.cone, eps_pri=1e-3, eps_dual=1e-3, eps_gap=1e-3, eps_infeas=1e-3,
                        eps_unbdd=1e-3, max_iters=args.solve_iters, time_limit_s=args.solve_seconds, **common)
        st3, _x, _y, _s, info3 = S3.solve()
        S3.close()
        torch.cuda.synchronize()
        tot = time.perf_counter() - t0
        paper_ctx = {"eps": 1e-3, "status": int(st3), "iters": info3["iters"], "seconds_total": tot,
                     "setup_s": info3["setup_s"], "solve_s": info3["solve_s"], "pobj": info3["pobj"],
                     "paper_gpu": dict(PAPER_APPS[args.workload][2], hardware="GeForce GTX Titan X (Maxwell), "
                                       "indirect method, cuSPARSE SpMV, setup included")}

    oerr = None
    if err_proc is not None:
        try:
            orc = err_q.get(timeout=900)
        except Exception as e:
            orc = {"error": "no result: " + repr(e)}
        err_proc.join(timeout=10)
        oerr = oracle_err(args.seed, orc, common)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "iter/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if prec == 0 else "f32",
            "data": "synthetic (Sec. 6.6 generator, seed %d)" % args.seed,
            "config": {"workload": desc,
                       "precision": "fp64 throughout" if prec == 0 else
                       "fp32 A, CG and working iterates; fp64 scaling, tau, tests and outputs",
                       "l2": ("inputs larger than L2 (A and A^T in CSR: %.0f MB)" % (2 * (4 + 4 * (2 - prec)) * P.A.nnz / 1e6)
                              if 2 * (4 + 4 * (2 - prec)) * P.A.nnz > 129e6 else
                              "inputs fit in L2 (a parity-size program: no flush, not a headline line)"),
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "step": "one ADMM iteration with the solve's Sec. 3.5 tests every 20 iterations",
                       "linsys": "direct (cached dense inverse)" if args.linsys else "indirect (PCG)",
                       "cg_steps_per_iter": cg_steps / max(it1 - it0, 1)},
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clk, "time_to_1e4": solve,
        }
        if oerr is not None:
            line["oracle_err"] = oerr
        if paper_ctx is not None:
            line["paper_context"] = paper_ctx
        if psd is not None:
            line["psd_roofline"] = psd
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


BATCH_DESC = ("{count} portfolio SOCPs (long-only factor model, Sec. 6.3 form with one risk SOC): n ~ U[20, 500] "
              "assets, k = n/10 factors, F ~ N(0,1), mu ~ U(0,1); zero 1, nonneg n, SOC k+2 per program")


BATCH_MAX_ITERS = 50000


def batch_programs(workload, seed):
    from paper_1312_3039_gb300 import synth
    count = 4096 if workload == "portfolio_batch" else 256
    progs = synth.portfolio_batch(seed, count=count)
    return progs, BATCH_DESC.format(count=count)


def cpu_batch_job(workload, seed, seconds, queue):
    """CPU baseline of a batched workload: the FP64 oracle (direct method,
    one thread) solving programs of a stratified sample for about `seconds`."""
    try:
        progs, _ = batch_programs(workload, seed)
        from oracle import admm
        order = sorted(range(len(progs)), key=lambda i: progs[i].n)
        pick = order[::max(1, len(order) // 64)]
        t0 = time.perf_counter()
        done = 0
        for i in pick:
            P = progs[i]
            admm.solve(P.A, P.b, P.c, P.cone, admm.Settings(max_iters=BATCH_MAX_ITERS))
            done += 1
            if time.perf_counter() - t0 >= seconds:
                break
        queue.put({"programs": done, "seconds": time.perf_counter() - t0, "of": len(pick)})
    except Exception as e:
        queue.put({"error": repr(e)})


def run_batch(args):
    """Batched workload: every program solved to the 1e-4 tests by one
    persistent launch (a CUDA graph) per step; the plain solver (scs_init +
    scs_solve per program) on a stratified sample gives the looped time."""
    world, rank, local = dist_env()
    cpu_proc = cpu_q = None
    if rank == 0 and not args.no_cpu_baseline:
        import multiprocessing as mp
        ctx = mp.get_context("spawn")
        cpu_q = ctx.Queue()
        cpu_proc = ctx.Process(target=cpu_batch_job, args=(args.workload, args.seed, args.cpu_seconds, cpu_q),
                               daemon=True)
        cpu_proc.start()
    import numpy as np
    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    from paper_1312_3039_gb300 import scs
    progs, desc = batch_programs(args.workload, args.seed)
    count = len(progs)
    tuples = [(P.A, P.b, P.c, P.cone) for P in progs]
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    # 50000 iterations at most: about 9% of the 4096 programs need more than
    # 10000 (the FP64 oracle as well; at most 37580)
    common = dict(precision=1, device=local, cuda_stream=stream.cuda_stream, max_iters=BATCH_MAX_ITERS)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def reduce(x, op):
        return reduce_scalar(x, op)

    # end to end: host CSC -> scs_batch_init (setup launch + autotuner) ->
    # scs_batch_solve -> x, y, s and infos on the host
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    bt = scs.Batch(tuples, **common)
    init_s = time.perf_counter() - t0
    xs, ys, ss, infos = bt.solve()
    torch.cuda.synchronize()
    e2e_s = reduce(time.perf_counter() - t0, "max")
    cfg = bt.config()
    for _ in range(max(0, args.warmup - 1)):
        bt.solve()
    # timed: `steps` cold batched solves (graph launch .. last program done)
    clocks = ClockSampler(local)
    clocks.start()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    dev_ms = 0.0
    for _ in range(args.steps):
        barrier()
        torch.cuda.synchronize()
        e0.record(stream)
        xs, ys, ss, infos = bt.solve()
        e1.record(stream)
        torch.cuda.synchronize()
        dev_ms += e0.elapsed_time(e1)
    clk = clocks.stop()
    bt.close()
    value, total, secs = replica_rate(count * args.steps, dev_ms / 1e3)
    ms = secs * 1e3
    st = np.array([f["status"] for f in infos])
    iters = np.array([f["iters"] for f in infos])
    cg = np.array([f["cg_iters"] for f in infos])
    # plain solver, one program at a time, on a stratified sample
    order = sorted(range(count), key=lambda i: progs[i].n)
    pick = order[::max(1, count // args.plain_sample)]
    plain_s = 0.0
    plain_status = []
    for i in pick:
        P = progs[i]
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        r = scs.solve(P.A, P.b, P.c, P.cone, **common)
        torch.cuda.synchronize()
        plain_s += time.perf_counter() - t1
        plain_status.append(int(r[0] == infos[i]["status"] and r[4]["iters"] == infos[i]["iters"]))
    plain_total = plain_s / len(pick) * count
    # algorithmic bytes of the products: per program, per iteration one A^T
    # product and 2 per CG step, and the product A z on every 20th iteration
    # (the first of the solve included); each streams A^'s CSR (8 B per
    # nonzero + 4 B per row) and gathers its input once
    byt = 0.0
    for i, P in enumerate(progs):
        per = (8.0 * P.A.nnz + 4.0 * (P.m + P.n) + 4.0 * (P.n + P.m)) / 2.0
        byt += per * (iters[i] + 2 * cg[i] + (iters[i] + 19) // 20)
    peak, peak_src = measured_hbm_peak()
    achieved = byt * args.steps / (ms / 1e3) / 1e9
    cpu = None
    if cpu_proc is not None:
        try:
            r = cpu_q.get(timeout=900)
        except Exception as e:
            r = {"error": "no result: " + repr(e)}
        cpu_proc.join(timeout=10)
        if "error" in r:
            cpu = {"value": None, "unit": "programs/s", "cores": 1, "kind": "oracle", "sample": r["error"]}
        else:
            cpu = {"value": r["programs"] / r["seconds"], "unit": "programs/s", "cores": 1, "kind": "oracle",
                   "sample": f"{r['programs']} of a stratified sample of {r['of']} programs solved to 1e-4 by the "
                             f"FP64 oracle (direct method, one thread) in {r['seconds']:.1f} s"}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "programs/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic (Sec. 6.3 portfolio form, seed %d)" % args.seed,
            "config": {"workload": desc, "precision": "fp32 A/CG/iterates, fp64 scaling and tests",
                       "step": "one batched solve of every program to the 1e-4 tests (cold start)",
                       "l2": "each program's A stays in L1/L2 while its CTA solves it (<= 200 KB)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "autotuned": cfg},
            "batched": {"programs": count, "solve_s": ms / args.steps / 1e3, "status_counts":
                        {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
                        "iters_mean": float(iters.mean()), "iters_max": int(iters.max()),
                        "cg_per_iter": float(cg.sum() / max(iters.sum(), 1)),
                        "plain_looped_s_est": plain_total, "plain_sample": len(pick),
                        "plain_sample_same_status_and_iters": sum(plain_status),
                        "speedup_vs_plain": plain_total / (ms / args.steps / 1e3),
                        "init_s": init_s},
            "roofline": {"bound": "hbm", "kernel": "batch solve_kernel (all products of all programs)",
                         "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                         "peak_source": peak_src, "traffic": None,
                         "note": "operands L2/L1-resident while a team works on them: HBM peak as denominator"},
            "cpu_baseline": cpu,
            "e2e": {"value": count / e2e_s, "unit": "programs/s", "seconds": e2e_s,
                    "h2d_bytes_per_step": float(sum(12 * P.A.nnz + 8 * (P.n + 1) + 8 * (P.m + P.n) for P in progs)),
                    "d2h_bytes_per_step": float(sum(8 * (P.n + 2 * P.m) for P in progs) + 120 * count),
                    "includes": "scs_batch_init (host CSC->CSR, H2D, setup launch, autotuner) + scs_batch_solve + "
                                "D2H of x, y, s, info"},
            "gpu_launches": args.steps,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


LASSO_DESC = ("parametric lasso family (Sec. 6.2 SOCP form): F 1000x400 N(0,1)/sqrt(1000), theta in R^64, "
              "g = G theta, mu = mu0 (1 + tanh(a.theta/8)/2); n=801 m=1802; network 64-512-512-512-4406 GELU, "
              "BF16; {train} training solves, {held} held-out members")


def run_lasso_warm(args):
    """Learned warm start: the family solver generates the training states,
    the network trains on them, and held-out members are solved cold and
    warm-started (inference, projection and warm start inside the timed
    warm solve); the plain solver (scs_solve per member) cold and warm on a
    sample of the held-out members."""
    world, rank, local = dist_env()
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    from paper_1312_3039_gb300 import scs, synth
    from paper_1312_3039_gb300.warmstart import LearnedWarmStart
    small = args.workload == "lasso_warm_small"
    ntrain = args.train or (4096 if small else 100000)
    nheld = 1024 if small else 10000
    fam = synth.lasso_family(args.seed)
    ws = LearnedWarmStart(fam, scs, torch, batch=1024, seed=args.seed)
    th_tr = fam.thetas(args.seed + 100, ntrain)
    th_te = fam.thetas(args.seed + 200, nheld)
    t0 = time.perf_counter()
    infos_tr, gen_s, states = ws.solve_family(th_tr)
    gen_wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    t1 = time.perf_counter()
    hist = ws.fit(th_tr, states, epochs=args.epochs, lr=1e-3)
    torch.cuda.synchronize()
    fit_s = time.perf_counter() - t1
    steps = args.epochs * (ntrain // ws.batch)
    flop_step = 6.0 * ws.batch * sum(a * b for a, b in zip(ws.sizes[:-1], ws.sizes[1:]))
    del states
    # held-out: warm-up solve, then `steps` timed cold and warm solves
    clocks = ClockSampler(local)
    ws.solve_family(th_te[:1024])
    clocks.start()
    cold_s, warm_s = 0.0, 0.0
    for _ in range(args.steps):
        cold, cs, _ = ws.solve_family(th_te)
        warm, wsec, _ = ws.solve_family(th_te, warm=ws.predict_warm)
        cold_s += cs
        warm_s += wsec
    clk = clocks.stop()
    ci = np.array([f["iters"] for f in cold])
    wi = np.array([f["iters"] for f in warm])
    # family solver: the three FP32 products of an iteration, 2 (nm + n^2 + mn)
    # flops per member, counted for each member's own iterations (members that
    # finished early are dropped from the products at the next compaction)
    nn, mm = fam.A.shape[1], fam.A.shape[0]
    fam_flops = float(ci.sum()) * 2.0 * (2.0 * nn * mm + nn * nn)
    fam_tflops = fam_flops / (cold_s / args.steps) / 1e12
    fp32_peak = fp32_alu_peak_tflops(clk.get("sm_mhz"))
    bf16_peak, bf16_src = 1900.0, "fallback"
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            bf16_peak, bf16_src = float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        pass
    # plain solver (scs_solve per member, indirect CG), cold and warm-started
    # from the network's prediction mapped to the caller's units
    pick = list(range(0, nheld, max(1, nheld // args.plain_sample)))
    xh, yh, sh = ws.predict_warm(th_te[pick])
    xh, yh, sh = xh.cpu().numpy(), yh.cpu().numpy(), sh.cpu().numpy()
    pc_s = pw_s = 0.0
    pci, pwi = [], []
    for k, i in enumerate(pick):
        P = fam.problem(th_te[i])
        with scs.Solver(P.A, P.b, P.c, P.cone, precision=1) as S:
            D, E, sg, rh = S.scaling()
            torch.cuda.synchronize()
            a = time.perf_counter()
            st, *_r, info = S.solve()
            pc_s += time.perf_counter() - a
            pci.append(info["iters"])
            a = time.perf_counter()
            S.warm_start(E * xh[k] / sg, D * yh[k] / rh, sh[k] / (sg * D))
            st2, *_r2, info2 = S.solve()
            pw_s += time.perf_counter() - a
            pwi.append(info2["iters"])
    ws.close()
    line = {
        "metric": METRIC, "value": args.steps * nheld / warm_s, "unit": "held-out members/s (warm-started)",
        "n_gpus": 1, "steps": args.steps, "warmup": 1, "ms_per_step": 1e3 * warm_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 solve, bf16 network",
        "data": "synthetic (Sec. 6.2 lasso form, seed %d)" % args.seed,
        "config": {"workload": LASSO_DESC.format(train=ntrain, held=nheld),
                   "step": "one family solve of every held-out member to the 1e-4 tests"},
        "warm_vs_cold": {"cold_s": cold_s / args.steps, "warm_s": warm_s / args.steps,
                         "time_ratio": warm_s / cold_s, "iters_cold_mean": float(ci.mean()),
                         "iters_warm_mean": float(wi.mean()), "iters_cold_median": float(np.median(ci)),
                         "iters_warm_median": float(np.median(wi)),
                         "warm_solved": float(np.mean([f["status"] == 1 for f in warm]))},
        "plain_solver_sample": {"members": len(pick), "cold_s": pc_s, "warm_s": pw_s,
                                "iters_cold_mean": float(np.mean(pci)), "iters_warm_mean": float(np.mean(pwi)),
                                "family_cold_s_same_members": cold_s / args.steps * len(pick) / nheld,
                                "family_warm_s_same_members": warm_s / args.steps * len(pick) / nheld},
        "training": {"members": ntrain, "generation_s": gen_s, "generation_wall_s": gen_wall, "fit_s": fit_s,
                     "epochs": args.epochs, "steps": steps, "loss_first_epoch": hist[0], "loss_last_epoch": hist[-1],
                     "train_tflops": flop_step * steps / fit_s / 1e12},
        # the FP32 family's products run on the tensor cores as six BF16
        # products per FP32 product (three-way split): tensor flops = 6 x the
        # FP32-equivalent flops, against the measured BF16 peak
        "roofline": {"bound": "tensor", "kernel": "family solver iteration (three FP32-accurate products over the "
                                                  "members, each six BF16 tcgen05 products of the split operands)",
                     "achieved": 6.0 * fam_tflops, "peak": bf16_peak, "unit": "TFLOP/s",
                     "frac": 6.0 * fam_tflops / bf16_peak, "peak_source": bf16_src,
                     "fp32_equivalent_tflops": fam_tflops, "fp32_alu_peak": fp32_peak,
                     "note": "over the whole family solve (the elementwise launches between the products included)",
                     "traffic": None},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_mlp_train(args):
    """The warm-start network alone: Adam steps of the 64-512-512-512-4406
    GELU network on a batch of 4096 (BF16 products, FP32 masters), on the
    tcgen05 and the mma.sync kernels, and one large product per kernel
    against the measured BF16 peak."""
    import numpy as np
    import torch
    from paper_1312_3039_gb300 import scs
    sizes = [64, 512, 512, 512, 4406]
    batch = 4096
    flop_step = 6.0 * batch * sum(a * b for a, b in zip(sizes[:-1], sizes[1:]))
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    rng = np.random.default_rng(args.seed)
    X = torch.randn(batch, 64, device="cuda")
    T = torch.randn(batch, 4406, device="cuda")
    res = {}
    clocks = ClockSampler(0)
    clocks.start()
    for tc in (1, 0):
        net = scs.MLP(64, 512, 3, 4406, batch, stream=stream.cuda_stream)
        params = [(rng.standard_normal((o, i)) / np.sqrt(i), np.zeros(o)) for i, o in zip(sizes[:-1], sizes[1:])]
        net.set_params(scs.pack_params(params))
        net.set_tensor_path(bool(tc))
        for _ in range(args.warmup):
            net.train_step(X.data_ptr(), T.data_ptr(), 1e-4)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            net.train_step(X.data_ptr(), T.data_ptr(), 1e-4)
        e1.record(stream)
        stream.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        assert net.error() == 0
        net.close()
        # one large product
        M, N, K = 16384, 4096, 4096
        A = torch.randn(M, K, dtype=torch.bfloat16, device="cuda")
        B = torch.randn(N, K, dtype=torch.bfloat16, device="cuda")
        C = torch.empty(M, N, dtype=torch.float32, device="cuda")
        for _ in range(3):
            scs.lib().scs_bf16_gemm(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C.data_ptr(), N, tc, stream.cuda_stream)
        # back-to-back launches (enqueue only), CUDA events on their stream
        err = torch.zeros(1, dtype=torch.int32, device="cuda")
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        stream.synchronize()
        g0.record(stream)
        R = 10
        for _ in range(R):
            rc = scs.lib().scs_bf16_gemm_async(A.data_ptr(), K, B.data_ptr(), K, M, N, K, C.data_ptr(), N, tc,
                                               err.data_ptr(), stream.cuda_stream)
            assert rc == 0, rc
        g1.record(stream)
        stream.synchronize()
        assert int(err.item()) == 0
        gms = g0.elapsed_time(g1) / R
        res[tc] = {"step_ms": ms, "step_tflops": flop_step / (ms / 1e3) / 1e12,
                   "gemm_ms": gms, "gemm_tflops": 2.0 * M * N * K / (gms / 1e3) / 1e12}
    clk = clocks.stop()
    peak = 1905.4
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peak = float(json.load(f)["bf16_tflops"])
        src = "measured"
    except Exception:
        src = "fallback"
    line = {
        "metric": METRIC, "value": batch / (res[1]["step_ms"] / 1e3), "unit": "training samples/s (tcgen05)",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": res[1]["step_ms"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16 products, fp32 accumulate",
        "data": "synthetic (random inputs and targets)",
        "config": {"workload": "warm-start network 64-512-512-512-4406 GELU, Adam, batch 4096",
                   "gemm": "16384 x 4096 x 4096 (C = A B^T), per kernel"},
        "paths": {"tcgen05": res[1], "mma_sync": res[0]},
        "roofline": {"bound": "tensor", "kernel": "gemm_nt_tc_kernel (tcgen05) 16384x4096x4096",
                     "achieved": res[1]["gemm_tflops"], "peak": peak, "unit": "TFLOP/s",
                     "frac": res[1]["gemm_tflops"] / peak, "peak_source": src + " (bf16 burst)", "traffic": None},
        "cpu_baseline": None, "e2e": None, "gpu_launches": None, "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.workload == "mlp_train":
        return run_mlp_train(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("portfolio_batch"):
        return run_batch(args)
    if args.workload.startswith("lasso_warm"):
        return run_lasso_warm(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
