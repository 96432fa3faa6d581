"""Benchmark of the reproducible Jacobi-PCG hot path on one GB300.

Headline: PCG iterations per second of the exblas variant on the 27-point
3D Poisson operator on a 256^3 grid (n = 16,777,216, nnz = 449,455,096,
FP64 CSR with int32 indices, Jacobi preconditioner, b = A x_true with
x_true ~ U[-1, 1], x0 = 0, tol 1e-8, at most 5000 iterations).  One step
is one complete solve (set-up plus every iteration until convergence);
value = iterations of the K timed solves / their device time.

Also reported on the same JSON line: the plain (non-reproducible,
tree-reduction) GPU PCG and the overhead ratio, the fpe variant's rate, the
exact dot's GB/s on 2^28-element U[-1, 1] pairs, the roofline of the
dominant kernel (pass A: SpMV + <d, w>), an end-to-end number through the
host-buffer C ABI, the CPU oracle timed on the host cores, and two
sub-records: the batched workload (256 variable-diffusion systems in one
launch sequence) and the serving workload (Poisson arrivals of 7-point
systems; capacity, 80% load and the offered 2000 req/s).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Under torchrun each rank solves its own copy of the system (the solve does
not shard across GPUs here: replicas only); value sums all ranks.
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

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synth  # noqa: E402

PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_HBM_GBS = 6800.0
METRIC = "PCG iters/s & overhead vs plain GPU PCG; exact-dot GB/s vs HBM peak (bit-exact)"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--side", type=int, default=256, help="grid side of the Poisson workload")
    ap.add_argument("--stencil", type=int, choices=[7, 27], default=27, help="7- or 27-point Poisson")
    ap.add_argument("--variant", choices=["exblas", "fpe", "plain"], default="exblas",
                    help="dot variant of the timed solves (the headline uses exblas)")
    ap.add_argument("--band", type=int, default=0, metavar="BW",
                    help="use the band matrix of half-bandwidth BW (the paper's performance workload) instead")
    ap.add_argument("--band-n", type=int, default=4_000_000, help="rows of the band matrix")
    ap.add_argument("--max-iter", type=int, default=5000)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true", help="skip the plain/fpe/dot/e2e side measurements")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched-workload record of the default line")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving record of the default line")
    ap.add_argument("--serve-window", type=float, default=15.0,
                    help="seconds per serving phase window in the default line's serving record")
    ap.add_argument("--serve", type=float, default=0.0, metavar="SECONDS",
                    help="only the serving workload: Poisson arrivals of 7-point systems, side log-uniform in [16,128]")
    ap.add_argument("--rate", type=float, default=2000.0, help="offered arrival rate for --serve (requests/s)")
    ap.add_argument("--batch", type=int, default=0, metavar="COUNT",
                    help="only the batched workload: COUNT variable-diffusion systems, s ~ U{8..64}, tol 1e-10")
    ap.add_argument("--dot-only", type=int, default=0, metavar="LOG2N",
                    help="only time the exact, fpe and plain dots on 2^LOG2N pairs of --dot-family")
    ap.add_argument("--dot-family", default="a", choices=["a", "b", "c8", "c16", "c24", "c32", "c40"],
                    help="pairs for --dot-only: (a) U[-1,1]; (b) m 2^e, e in [-300, 300]; (cK) cond 1eK")
    ap.add_argument("--eager", action="store_true",
                    help="launch the solver's kernels one by one instead of the graph (for profilers)")
    return ap.parse_args()


def hbm_peak():
    try:
        with open(PEAKS_FILE) as f:
            return float(json.load(f)["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def workload(side, stencil=27, band=0, band_n=0):
    if band:
        A = synth.band(band_n, band)
    else:
        A = synth.poisson27(side) if stencil == 27 else synth.poisson7(side)
    xt = synth.poisson_rhs_xtrue(A.n, synth.BASE_SEED + 2)
    return A, xt


# DRAM traffic of one pass-A launch (dram__bytes_read.sum + write.sum), from
# the ncu captures summarised in profiles/k_pass_a_p27_128.md: the 27-point
# 256^3 launch measured at full size (a one-pass metric), and for other
# 27-point sizes the 128^3 launch's ratio to its algorithmic bytes (the
# kernel streams every matrix entry once).
PASS_A_TRAFFIC_256 = 5613844480 + 112287488
PASS_A_TRAFFIC_RATIO = 702.0 / 710.9


def pass_a_traffic(args, n, nnz):
    """(bytes, source) of one pass-A launch's DRAM traffic for the roofline
    record: measured at 27-point 256^3, scaled from 128^3 for other 27-point
    sizes, None for workloads no capture covers."""
    if args.band or args.stencil != 27:
        return None, None
    if args.side == 256:
        return PASS_A_TRAFFIC_256, "ncu dram bytes of the 27-point 256^3 pass A launch, measured at full size"
    return (PASS_A_TRAFFIC_RATIO * pass_a_bytes(n, nnz),
            "ncu dram bytes of the 27-point 128^3 launch scaled by algorithmic bytes")


# Pipe utilisation of the fpe variant's three FPE-dot kernels, from the ncu
# full-set capture summarised in profiles/k_fpe_dots_p27_128.md (27-point
# 128^3, percent of each pipe's own peak while the SMs are active).  The
# FP64 pipe, half rate on this GPU, is the busiest unit: the fpe roof.
FPE_PIPES = {"k_pass_a_dot": {"fp64": 52.1, "alu": 62.0, "issue": 61.3},
             "k_pass_b1": {"fp64": 62.9, "alu": 54.3, "issue": 55.2},
             "k_pass_b2": {"fp64": 53.3, "alu": 61.0, "issue": 61.6}}


def wl_name(args):
    return f"band_{args.band_n}_bw{args.band}" if args.band else f"poisson{args.stencil}_{args.side}"


def pass_a_bytes(n, nnz):
    """Algorithmic bytes of one pass-A launch: CSR stream, d read once, w written once."""
    return 12 * nnz + 4 * (n + 1) + 8 * n + 8 * n


def iter_bytes(n, nnz):
    """Algorithmic bytes of one PCG iteration (three passes, z recomputed)."""
    return 12 * nnz + 4 * (n + 1) + 88 * n


def l2_note(n, nnz):
    """How the timed inputs relate to the 129 MB L2 (the timing rule)."""
    csr = 12 * nnz + 4 * (n + 1)
    if csr > (129 << 20):
        return f"inputs larger than L2 (CSR {csr / 1e9:.2f} GB streamed every iteration)"
    return (f"inputs fit in L2 (CSR {csr / 1e6:.2f} MB): a latency-bound workload, timed warm as a solver "
            "sees it between iterations")


def small_system_rates(P, dev, stream, steps=20):
    """7-point Poisson 16^3 (4096 rows), b = A x_true, tol 1e-8: iterations/s
    of complete solves for each variant, and the path rpcg_solve takes."""
    import torch
    A, xt = workload(16, 7, 0, 0)
    M = P.Matrix.from_csr(A)
    b = M.spmv(torch.from_numpy(xt).to(dev))
    x = torch.zeros(A.n, dtype=torch.float64, device=dev)
    out = {}
    for v, k in (("exblas", steps), ("plain", steps), ("fpe", steps)):
        for _ in range(3):
            x.zero_()
            r = M.solve(b, x, variant=v, tol=1e-8, max_iter=1000)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        it = 0
        e0.record(stream)
        for _ in range(k):
            x.zero_()
            r = M.solve(b, x, variant=v, tol=1e-8, max_iter=1000)
            it += r["iterations"]
        e1.record(stream)
        torch.cuda.synchronize()
        out[v] = {"iters_per_s": it / (e0.elapsed_time(e1) / 1e3), "iterations": r["iterations"],
                  "status": r["status"], "path": M.solve_path(v)}
    out["overhead_exblas_vs_plain"] = out["plain"]["iters_per_s"] / out["exblas"]["iters_per_s"]
    out["overhead_fpe_vs_plain"] = out["plain"]["iters_per_s"] / out["fpe"]["iters_per_s"]
    out["workload"] = "poisson7_16 (n 4096, nnz 27136), b = A x_true, tol 1e-8, complete solves from x0 = 0"
    return out


def family_c_dot_record(P, dev, stream, peak):
    """Exact dot of ill-conditioned family-(c) pairs (target condition number
    1e32; the realised one, 2 sum|a_i b_i| / |a . b|, is reported), a 2^24
    draw tiled 4x to 2^26 pairs (1.07 GB, larger than L2).  Its bit-exactness
    against the oracle is a full-size test (tests/test_gpu_fullsize.py)."""
    import torch
    base = 1 << 24
    a, b = synth.dot_family_c(base, 1e32, synth.BASE_SEED + 5)
    da = torch.from_numpy(a).to(dev).repeat(4)
    db = torch.from_numpy(b).to(dev).repeat(4)
    out = torch.empty((), dtype=torch.float64, device=dev)
    for _ in range(3):
        P.dot_exact(da, db, out=out)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        P.dot_exact(da, db, out=out)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    n = 4 * base
    v = out.item()
    rec = {"n": n, "cond_target": 1e32, "ms": ms, "gbs": 16 * n / (ms * 1e-3) / 1e9,
           "frac": 16 * n / (ms * 1e-3) / 1e9 / peak,
           "cond_realised": 2.0 * float(torch.sum(torch.abs(da) * torch.abs(db)).item()) / abs(v)}
    return rec


def reduce_over_ranks(v, op, device):
    """Max or sum of a scalar over the ranks of the default process group
    (identity without one).  Timings take the max, work counts the sum."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return v
    t = torch.tensor([float(v)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return float(t.item())


class ClockSampler:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region."""

    FIELDS = "clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown," \
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown," \
             "clocks_event_reasons.sw_power_cap"

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.out = None

    def start(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "200"], stdout=self.out,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.out.flush()
        self.out.seek(0)
        rows = [ln.strip().split(", ") for ln in self.out.read().splitlines() if ln.strip()]
        os.unlink(self.out.name)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[0]))
                mx = float(r[1])
                for nm, v in zip(names, r[3:7]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except Exception:
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- CPU oracle leg

def cpu_oracle_rate(A, b, iters, tol, nthreads=None):
    """The oracle as it stands, on all host cores (or nthreads): iterations
    per second of its PCG loop (set-up excluded) over a bounded number of
    iterations."""
    import oracle
    nt = oracle.default_threads() if nthreads is None else nthreads
    r = oracle.pcg(A, b, variant=oracle.EXACT, tol=tol, max_iter=iters, nthreads=nt)
    return r["iterations"] / max(r["loop_seconds"], 1e-9), r["iterations"], r["loop_seconds"], nt


def workload_config(args, n, nnz):
    """The workload both arms measure (the reference arm's config equals this one)."""
    return {"workload": wl_name(args) + " " + args.variant, "n": n, "nnz": nnz, "tol": args.tol,
            "max_iter": args.max_iter, "l2": l2_note(n, nnz), "parallelism": f"replicas x{args.gpus}",
            "metric_unit": "PCG iterations (loop bodies) per second"}


def reference_arm(args, rank, world):
    """--impl reference: the CPU oracle, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    import oracle
    A, xt = workload(args.side, args.stencil, args.band, args.band_n)
    b = oracle.spmv(A, xt, nthreads=oracle.default_threads())
    per_step = 2
    for _ in range(args.warmup):
        cpu_oracle_rate(A, b, 1, args.tol)
    its, secs = 0, 0.0
    nt = 1
    for _ in range(args.steps):
        _, it, s, nt = cpu_oracle_rate(A, b, per_step, args.tol)
        its += it
        secs += s
    v = its / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "iters/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(args, A.n, A.nnz),
            "run": {"step": f"{per_step} PCG iterations of the oracle on the host cores (set-up excluded "
                            "from the time); the exact-dot trajectory the exblas variant follows"},
            "cpu_baseline": {"value": v, "unit": "iters/s", "cores": nt, "kind": "oracle",
                             "sample": f"{args.steps} x {per_step} iterations of the exact-dot PCG"},
            "e2e": {"value": v, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- GPU leg

def gpu_arm(args, rank, world, local_rank):
    import torch

    import paper_2005_07282_gb300 as P
    from paper_2005_07282_gb300 import build as B

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    B.build()
    dist = None
    if world > 1:
        import torch.distributed as dist
    stream = torch.cuda.current_stream()

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return reduce_over_ranks(v, "max", dev)

    def sum_over_ranks(v):
        return reduce_over_ranks(v, "sum", dev)

    # ---- inputs (host CSR in pinned memory for the end-to-end leg)
    A, xt = workload(args.side, args.stencil, args.band, args.band_n)
    n, nnz = A.n, A.nnz
    M = P.Matrix.from_csr(A)
    d_xt = torch.from_numpy(xt).to(dev)
    d_b = M.spmv(d_xt)
    torch.cuda.synchronize()
    x = torch.zeros(n, dtype=torch.float64, device=dev)
    opts = dict(tol=args.tol, max_iter=args.max_iter)

    def solve(variant, **kw):
        x.zero_()
        if args.eager:
            return M.solve_profiled(d_b, x, variant=variant, **{**opts, **kw})
        return M.solve(d_b, x, variant=variant, **{**opts, **kw})

    # ---- warm-up (builds and caches the graphs)
    for _ in range(args.warmup):
        r = solve(args.variant)
    iters_per_solve = r["iterations"]
    status = r["status"]

    # ---- timed region: K full exblas solves
    clocks = ClockSampler(local_rank)
    clocks.start()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    total_iters = 0
    for _ in range(args.steps):
        r = solve(args.variant)
        total_iters += r["iterations"]
    e1.record(stream)
    barrier()
    ms = e0.elapsed_time(e1)
    clk = clocks.stop()
    ms_max = max_over_ranks(ms)
    all_iters = sum_over_ranks(total_iters)
    value = all_iters / (ms_max / 1e3)
    path = "graph" if args.eager else M.solve_path(args.variant)
    # our kernels per timed solve: one cluster launch, or the graph's set-up
    # kernels plus passes A, B, C per iteration
    launches = args.steps * (1 if path == "cluster" else 4 + 3 * iters_per_solve)

    extras = {}
    cpu = None
    roof = None
    e2e = None
    if not args.no_extras:
        # plain GPU PCG (tree-reduction dots): the overhead baseline
        rp = solve("plain")
        torch.cuda.synchronize()
        e0.record(stream)
        pit = 0
        for _ in range(args.steps):
            rp = solve("plain")
            pit += rp["iterations"]
        e1.record(stream)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1)
        plain_rate = pit / (pms / 1e3)
        extras["plain_iters_per_s"] = plain_rate
        extras["plain_iterations"] = rp["iterations"]
        extras["overhead_vs_plain"] = plain_rate / (total_iters / (ms / 1e3))
        # fpe variant (FPE8 with early exit; FP64-pipe bound on this GPU), bounded iterations
        fit = min(100, iters_per_solve)
        solve("fpe", max_iter=5)
        torch.cuda.synchronize()
        e0.record(stream)
        rf = solve("fpe", max_iter=fit)
        e1.record(stream)
        torch.cuda.synchronize()
        extras["fpe_iters_per_s"] = rf["iterations"] / (e0.elapsed_time(e1) / 1e3)
        extras["fpe_sample_iterations"] = rf["iterations"]
        # the paper's Poisson sweet spot (FPE3) and the adaptive size
        for label, fs in (("fpe3", 3), ("fpe_adaptive", 0)):
            e0.record(stream)
            rr = solve("fpe", max_iter=fit, fpe_size=fs)
            e1.record(stream)
            torch.cuda.synchronize()
            extras[f"{label}_iters_per_s"] = rr["iterations"] / (e0.elapsed_time(e1) / 1e3)
            extras[f"{label}_inexact_dots"] = rr["fpe_inexact_count"]
            extras[f"{label}_size_used"] = rr["fpe_size_used"]
        # per-pass event timing (same kernels launched one by one), bounded iterations
        x.zero_()
        prof = M.solve_profiled(d_b, x, variant="exblas", tol=args.tol, max_iter=min(60, iters_per_solve))
        la = prof["launches"]["A"]
        a_ms = prof["pass_ms"]["A"] / max(la, 1)
        b_ms = prof["pass_ms"]["B"] / max(la, 1)
        c_ms = prof["pass_ms"]["C"] / max(la, 1)
        peak, peak_kind = hbm_peak()
        ach = pass_a_bytes(n, nnz) / (a_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": pass_a_traffic(args, n, nnz)[0],
                "traffic_source": pass_a_traffic(args, n, nnz)[1],
                "kernel": "k_pass_a (SpMV + <d,w> exact deposit)",
                "peak_kind": f"{peak_kind} copy bandwidth",
                "algorithmic_bytes_per_launch": pass_a_bytes(n, nnz), "avg_launch_ms": a_ms}
        extras["pass_ms"] = {"A": a_ms, "B": b_ms, "C": c_ms}
        x.zero_()
        pf = M.solve_profiled(d_b, x, variant="fpe", tol=args.tol, max_iter=min(30, iters_per_solve))
        lf = max(pf["launches"]["A"], 1)
        extras["pass_ms_fpe"] = {k: pf["pass_ms"][k] / lf for k in ("A", "B", "C")}
        fpe_ms = 1e3 / extras["fpe_iters_per_s"]
        extras["fpe_roofline"] = {
            "bound": "issue (FP64 and ALU pipes each 52-63% busy)",
            "kernels": "k_pass_a_dot, k_pass_b1, k_pass_b2 (the iteration's three FPE dots)",
            "pipe_active_pct": FPE_PIPES, "source": "ncu --set full, 27-point 128^3 (profiles/k_fpe_dots_p27_128.md)",
            "iteration_ms": fpe_ms, "iteration_hbm_frac": iter_bytes(n, nnz) / (fpe_ms * 1e-3) / 1e9 / hbm_peak()[0],
            "overhead_vs_plain": plain_rate / extras["fpe_iters_per_s"]}
        it_ms = ms / max(total_iters, 1)
        extras["iteration_roofline"] = {"bytes_per_iter": iter_bytes(n, nnz), "ms_per_iter": it_ms,
                                        "achieved_gbs": iter_bytes(n, nnz) / (it_ms * 1e-3) / 1e9,
                                        "frac": iter_bytes(n, nnz) / (it_ms * 1e-3) / 1e9 / peak}
        # exact dot GB/s: 2^28 U[-1,1] pairs (a 2^24 draw tiled 16x in HBM)
        nd = 1 << 28
        base_a, base_b = synth.dot_family_a(1 << 24, synth.BASE_SEED + 1)
        da = torch.from_numpy(base_a).to(dev).repeat(16)
        db = torch.from_numpy(base_b).to(dev).repeat(16)
        out = torch.empty((), dtype=torch.float64, device=dev)
        for _ in range(3):
            P.dot_exact(da, db, out=out)
        torch.cuda.synchronize()
        e0.record(stream)
        reps = 10
        for _ in range(reps):
            P.dot_exact(da, db, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        dms = e0.elapsed_time(e1) / reps
        gbs = 16 * nd / (dms * 1e-3) / 1e9
        e0.record(stream)
        for _ in range(reps):
            P.dot_plain(da, db)
        e1.record(stream)
        torch.cuda.synchronize()
        pgbs = 16 * nd / (e0.elapsed_time(e1) / reps * 1e-3) / 1e9
        extras["exact_dot"] = {"n": nd, "gbs": gbs, "frac": gbs / peak, "ms": dms, "plain_dot_gbs": pgbs,
                               "inputs": "U[-1,1] pairs, 2^24 draw tiled 16x (4.3 GB, larger than L2)"}
        del da, db
        extras["exact_dot"]["family_c"] = family_c_dot_record(P, dev, stream, peak)
        # the small-system configuration (7-point 16^3, tol 1e-8): every variant
        if not (args.stencil == 7 and args.side == 16 and not args.band):
            extras["small_system"] = small_system_rates(P, dev, stream)
        # end to end through the host-buffer ABI: create from pinned host CSR, solve_host, destroy
        h_rowptr = torch.from_numpy(A.rowptr).pin_memory()
        h_col = torch.from_numpy(A.col).pin_memory()
        h_val = torch.from_numpy(A.val).pin_memory()
        h_b = d_b.cpu().pin_memory()
        h_x = torch.zeros(n, dtype=torch.float64).pin_memory()
        e2e_steps = max(1, min(args.steps, 2))
        t0 = time.perf_counter()
        eit = 0
        for _ in range(e2e_steps):
            M2 = P.Matrix(h_rowptr.numpy(), h_col.numpy(), h_val.numpy(), n=n)
            h_x.zero_()
            re = M2.solve_host(h_b.numpy(), h_x.numpy(), variant="exblas", **opts)
            eit += re["iterations"]
            M2.close()
        torch.cuda.synchronize()
        et = time.perf_counter() - t0
        e2e = {"value": sum_over_ranks(eit) / max_over_ranks(et), "unit": "iters/s",
               "h2d_bytes_per_step": int(12 * nnz + 4 * (n + 1) + 16 * n), "d2h_bytes_per_step": int(8 * n + 64),
               "path": "rpcg_create(host CSR) + rpcg_solve_host + rpcg_destroy"}
        del M2
        if rank == 0 and not args.no_cpu_baseline:
            import oracle
            b_host = d_b.cpu().numpy()
            crate, cit, csec, cores = cpu_oracle_rate(A, b_host, 3, args.tol)
            srate, sit, ssec, _ = cpu_oracle_rate(A, b_host, 1, args.tol, nthreads=1)
            cpu = {"value": crate, "unit": "iters/s", "cores": cores, "kind": "oracle",
                   "sample": f"{cit} exact-dot PCG iterations of the same system ({csec:.1f} s, set-up excluded)",
                   "single_thread": {"value": srate, "sample": f"{sit} iteration on one core ({ssec:.1f} s)"}}
        # the batched and serving workloads (rank 0; each GPU of a replica run would do the same)
        if rank == 0 and not args.no_batch:
            extras["batch"] = batch_record(P, dev, 256, "exblas", steps=3, warmup=2)
        if rank == 0 and not args.no_serve:
            extras["serving"] = serving_record(P, dev, args.serve_window, args.rate, 1.0)

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "iters/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": workload_config(args, n, nnz),
                "run": {"iterations_per_solve": iters_per_solve, "solve_status": status,
                        "step": "one complete solve from x0 = 0",
                        "launch": "eager (kernel by kernel)" if args.eager else
                        ("one cluster-resident launch per solve" if path == "cluster" else
                         "CUDA graph, device-side loop")},
                "roofline": roof, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, **extras}
        print(json.dumps(line), flush=True)


def dot_arm(args):
    """--dot-only: the three dot products on 2^k pairs of one family (16 B per
    element; a draw of at most 2^24 pairs, tiled)."""
    import torch

    import paper_2005_07282_gb300 as P
    from paper_2005_07282_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    n = 1 << args.dot_only
    base = min(n, 1 << 24)
    fam = args.dot_family
    if fam.startswith("c"):
        a0, b0 = synth.dot_family_c(base, float("1e" + fam[1:]), synth.BASE_SEED + 5)
    else:
        a0, b0 = getattr(synth, f"dot_family_{fam}")(base, synth.BASE_SEED + 1)
    da = torch.from_numpy(a0).to(dev).repeat(n // base)
    db = torch.from_numpy(b0).to(dev).repeat(n // base)
    peak, kind = hbm_peak()
    res = {}
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, fn in (("exact", lambda: P.dot_exact(da, db)), ("fpe", lambda: P.dot_fpe(da, db)),
                     ("plain", lambda: P.dot_plain(da, db))):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        res[name] = {"ms": ms, "gbs": 16 * n / (ms * 1e-3) / 1e9, "frac": 16 * n / (ms * 1e-3) / 1e9 / peak}
    print(json.dumps({"workload": f"dot family {fam} n=2^{args.dot_only}", "peak_gbs": peak, "peak_kind": kind,
                      "steps": args.steps, "warmup": args.warmup, **res}), flush=True)


def batch_record(P, dev, count=256, variant="exblas", steps=3, warmup=2, max_iter=5000, eager=False):
    """The batched workload: `count` variable-diffusion 7-point systems, s ~
    U{8..64}, b ~ U[-1, 1], tol 1e-10, solved in one batched launch sequence
    per step; against solving the same systems one after the other, with the
    count of systems whose result is bit-identical to their solo solve."""
    import torch

    t0 = time.perf_counter()
    mats, rhs = synth.diffusion_batch(count, synth.BASE_SEED + 3)
    gen_s = time.perf_counter() - t0
    Ms = [P.Matrix.from_csr(A) for A in mats]
    bs = [torch.from_numpy(b).to(dev) for b in rhs]
    xs = [torch.zeros(A.n, dtype=torch.float64, device=dev) for A in mats]
    opts = dict(tol=1e-10, max_iter=max_iter)
    Bt = P.Batch(Ms)
    if eager:
        Bt.solve(bs, xs, variant=variant, **opts)  # autotune once (graph form), then time pass by pass

    def run():
        for x in xs:
            x.zero_()
        if eager:  # kernel by kernel (profilers see every launch)
            return Bt.solve_profiled(bs, xs, variant=variant, **opts)[0]
        return Bt.solve(bs, xs, variant=variant, **opts)

    for _ in range(warmup):
        res = run()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        res = run()
    e1.record()
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    its = [r["iterations"] for r in res]
    batch_x = [x.cpu().numpy().copy() for x in xs]
    # the same systems solved one by one (graph per system), and the bit check
    for x in xs:
        x.zero_()
    torch.cuda.synchronize()
    e0.record()
    solo = [M.solve(b, x, variant=variant, **opts) for M, b, x in zip(Ms, bs, xs)]
    e1.record()
    torch.cuda.synchronize()
    solo_ms = e0.elapsed_time(e1)
    n_same = sum(int(np.array_equal(a.view(np.int64), x.cpu().numpy().view(np.int64)) and
                     r["iterations"] == s_["iterations"]) for a, x, r, s_ in zip(batch_x, xs, res, solo))
    rows = sum(A.n for A in mats)
    nnz = sum(A.nnz for A in mats)
    blk, tile = Bt.tuned()
    for x in xs:
        x.zero_()
    _, pass_ms, pass_launches = Bt.solve_profiled(bs, xs, variant=variant, **opts)
    moved = sum(r["iterations"] * iter_bytes(A.n, A.nnz) for r, A in zip(res, mats))
    # rows still iterating at every 40th iteration (the shrinking active set)
    active_rows = {k: sum(A.n for r, A in zip(res, mats) if r["iterations"] > k) for k in range(0, max(its), 40)}
    peak, peak_kind = hbm_peak()
    Bt.close()
    for M in Ms:
        M.close()
    return {"workload": f"batch of {count} diffusion7 systems, s~U{{8..64}}, tol 1e-10, {variant}",
            "rows": rows, "nnz": nnz, "solves_per_s": count / (ms / 1e3), "ms_per_batch": ms,
            "iterations": {"total": sum(its), "min": min(its), "max": max(its), "mean": sum(its) / len(its)},
            "system_iters_per_s": sum(its) / (ms / 1e3),
            "algorithmic_bytes_per_batch": moved, "active_rows_by_iteration": active_rows,
            "achieved_gbs": moved / (ms * 1e-3) / 1e9,
            "roofline_frac": moved / (ms * 1e-3) / 1e9 / peak, "peak_kind": peak_kind,
            "sequential_solo_ms": solo_ms, "speedup_vs_sequential": solo_ms / ms,
            "bit_identical_to_solo": n_same == count, "systems_bit_identical_to_solo": n_same,
            "statuses": sorted(set(r["status"] for r in res)),
            "autotuned": {"block": blk, "tile": tile},
            "pass_ms_eager": {k: round(v, 3) for k, v in pass_ms.items()},
            "pass_launches_eager": pass_launches, "timed_eager": bool(eager),
            "steps": steps, "warmup": warmup, "generation_s": gen_s}


def batch_arm(args):
    """--batch COUNT: one batched solve of COUNT systems per step (--variant,
    exblas by default; tol 1e-10), against solving the same systems one after
    the other."""
    import torch

    import paper_2005_07282_gb300 as P
    from paper_2005_07282_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    print(json.dumps(batch_record(P, dev, args.batch, args.variant, args.steps, args.warmup, args.max_iter,
                                  args.eager)), flush=True)


def serving_record(P, dev, window_s=15.0, rate=2000.0, offered_window_s=1.0):
    """The serving workload: 7-point Poisson systems with side log-uniform in
    [16, 128] and b ~ U[-1, 1], exblas, tol 1e-8, under a 64 GB HBM budget;
    the 113 operators are registered with the server once.  Three phases:
    capacity (closed loop with every slot busy, `window_s`), open-loop
    Poisson arrivals at 80% of that capacity (`window_s`), and open-loop
    arrivals at the offered rate for `offered_window_s` (then drained).
    Reports solves/s and p50/p99 of queueing, service and total latency per
    phase, and checks a sample of results bit for bit against solving each
    system alone."""
    import threading

    import torch

    seed = synth.BASE_SEED + 4
    rng = np.random.default_rng(seed)
    t0 = time.perf_counter()
    mats = {s: synth.poisson7(s) for s in range(16, 129)}
    pool = synth.uniform_pm1(synth.stream_seed(seed, 1), 128 ** 3 + (1 << 20))
    gen_s = time.perf_counter() - t0

    srv = P.Server(hbm_budget_bytes=64 << 30, max_slots=256)
    ids = {s: srv.register(A) for s, A in mats.items()}

    def make_request():
        side = int(round(np.exp(rng.uniform(np.log(16), np.log(128)))))
        off = int(rng.integers(0, 1 << 20))
        return side, pool[off:off + mats[side].n]

    def pct(v, q):
        return float(np.percentile(np.asarray(v), q)) if v else None

    def phase(duration, rate=None, closed=0):
        """Open loop at `rate` for `duration` s, or a closed loop keeping
        `closed` requests in flight.  Returns throughput and latencies."""
        lat, qs, ss, statuses, sample = [], [], [], [], []
        lock = threading.Lock()
        done_count = [0]
        t_start = time.perf_counter()
        stop_at = t_start + duration
        moved = [0]

        def collect(t, ts_submit, req):
            x, r = srv.wait(t)
            now = time.perf_counter()
            A = mats[req[0]]
            with lock:
                moved[0] += r["iterations"] * iter_bytes(A.n, A.nnz)
                lat.append((now - ts_submit) * 1e6)
                qs.append(r["queue_us"])
                ss.append(r["service_us"])
                statuses.append(r["status"])
                done_count[0] += 1
                if len(sample) < 12 and A.n <= 64 ** 3:
                    sample.append((req, x.copy(), r["iterations"]))

        collectors = []
        if closed:
            inflight = threading.Semaphore(closed)

            def run_one(req, ts):
                try:
                    t = srv.submit_registered(ids[req[0]], req[1], tol=1e-8, max_iter=5000)
                    collect(t, ts, req)
                finally:
                    inflight.release()

            while time.perf_counter() < stop_at:
                inflight.acquire()
                req = make_request()
                th = threading.Thread(target=run_one, args=(req, time.perf_counter()))
                th.start()
                collectors.append(th)
        else:
            next_t = t_start
            while True:
                next_t += rng.exponential(1.0 / rate)
                if next_t >= stop_at:
                    break
                delay = next_t - time.perf_counter()
                if delay > 0:
                    time.sleep(delay)
                req = make_request()
                ts = time.perf_counter()
                t = srv.submit_registered(ids[req[0]], req[1], tol=1e-8, max_iter=5000)
                th = threading.Thread(target=collect, args=(t, ts, req))
                th.start()
                collectors.append(th)
        for th in collectors:
            th.join()
        wall = time.perf_counter() - t_start
        peak, _ = hbm_peak()
        return {"requests": done_count[0], "wall_s": wall, "solves_per_s": done_count[0] / wall,
                "achieved_gbs": moved[0] / wall / 1e9, "roofline_frac": moved[0] / wall / 1e9 / peak,
                "latency_us": {"p50": pct(lat, 50), "p99": pct(lat, 99)},
                "queue_us": {"p50": pct(qs, 50), "p99": pct(qs, 99)},
                "service_us": {"p50": pct(ss, 50), "p99": pct(ss, 99)},
                "statuses": sorted(set(statuses))}, sample

    cap, sample = phase(window_s, closed=256)
    capacity = cap["solves_per_s"]
    at80, s2 = phase(window_s, rate=0.8 * capacity)
    offered, s3 = phase(offered_window_s, rate=rate)
    # bit-identity of served results with solving each system alone
    checked, same = 0, 0
    for (side, b), x, its in (sample + s2)[:16]:
        A = mats[side]
        M = P.Matrix.from_csr(A)
        xd = torch.zeros(A.n, dtype=torch.float64, device=dev)
        r = M.solve(torch.from_numpy(np.ascontiguousarray(b)).to(dev), xd, variant="exblas", tol=1e-8, max_iter=5000)
        checked += 1
        same += int(r["iterations"] == its and np.array_equal(xd.cpu().numpy().view(np.int64), x.view(np.int64)))
        M.close()
    st = srv.stats()
    srv.close()
    return {"workload": "serving: 7-point Poisson, side log-uniform [16,128], b~U[-1,1], exblas, tol 1e-8, "
                        "64 GB budget, 256 slots, 113 registered operators",
            "window_s": window_s, "capacity_closed_loop": cap,
            "at_80pct_capacity": {"rate": 0.8 * capacity, **at80},
            "at_offered_rate": {"rate": rate, "arrival_window_s": offered_window_s, **offered},
            "bit_identical_to_alone_sample": same == checked, "sample_checked": checked,
            "server_stats": st, "generation_s": gen_s}


def serve_arm(args):
    """--serve SECONDS: the serving workload alone, SECONDS per phase window."""
    import torch

    import paper_2005_07282_gb300 as P
    from paper_2005_07282_gb300 import build as B
    B.build()
    dev = torch.device("cuda", 0)
    print(json.dumps(serving_record(P, dev, args.serve, args.rate, min(args.serve, 1.0))), flush=True)


def main():
    args = parse()
    if args.serve:
        serve_arm(args)
        return
    if args.batch:
        batch_arm(args)
        return
    if args.dot_only:
        dot_arm(args)
        return
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        reference_arm(args, rank, world)
        return
    if world > 1:
        import torch
        import torch.distributed as dist
        torch.cuda.set_device(local_rank)
        dist.init_process_group("nccl")
    try:
        gpu_arm(args, rank, world, local_rank)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
