"""Benchmark: multi-shift CG solve of the 24^4 SU(3) staggered operator
exported as block-CSR (3x3 complex blocks, 331,776 block rows, 33 blocks per
row), m = 0.05, eps = 0.8, 15 shifts log-spaced 1e-4..10, one Gaussian
right-hand side, tolerance 1e-10 on the FP64 true residual of every shift,
FP32 bulk with FP64 reliable updates every 50 iterations.

One step = one complete solve (every shift to tolerance). Reported:
  value      algorithmic HBM GB/s of the whole solve (bytes the executed
             kernels must move at minimum, see `solve_bytes`) / device time;
  e2e        the same through the C ABI with host source and solution
             buffers (copies inside the timed region);
  time_to_solution_ms, iterations, and the same solve in plain FP64;
  roofline   the block-CSR SpMV kernel: algorithmic bytes per launch /
             its mean launch time, sampled live with CUDA events on the
             solve's stream during the timed steps;
  cpu_baseline  the FP64 CPU oracle on a bounded sample of the workload.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank solves its own replica of the workload
(the solve does not shard); value sums the ranks' bytes over the max time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "multi-shift CG HBM GB/s & time-to-solution (all shifts) vs plain FP64 path"
WORKLOAD = "24^4 SU(3) staggered A=M^dag M as block-CSR, 15 shifts 1e-4..10, 1 RHS, mixed FP32/FP64"
L2_BYTES = 129 * 2 ** 20


SPMV_COUNTERS = os.path.join(ROOT, "profiles", "bsr_spmv_24x4_counters.md")
# the profiled kernel: its own text in bsr.cu (from its leading comment to
# the next launcher template) and the two headers it depends on
SPMV_HEADERS = ("common.cuh", "engine.h")
SPMV_KERNEL = ("bsr.cu", "// The FP32 PASS_A of a single system",
               "template <class T, int BD, int KIND, class TO>\nstatic void launch_one(")


def _code_only(text):
    """C/C++ source without comments and whitespace (what the compiler sees)."""
    import re
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return re.sub(r"\s+", "", text)


def spmv_source_hash(read=None):
    """Hash of the profiled kernel's code: its own text in bsr.cu (from its
    leading comment to the next launcher template) and the headers it depends
    on, comments and whitespace removed. `read(name)` returns a source file's
    text (default: the working tree)."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1102_2143_gb300", "csrc")
    if read is None:
        def read(name):
            with open(os.path.join(csrc, name)) as f:
                return f.read()
    h = hashlib.sha256()
    for name in SPMV_HEADERS:
        h.update(_code_only(read(name)).encode())
    src = read(SPMV_KERNEL[0])
    a = src.index(SPMV_KERNEL[1])
    h.update(_code_only(src[a:src.index(SPMV_KERNEL[2], a)]).encode())
    return h.hexdigest()


def load_spmv_traffic():
    """DRAM bytes (read + write) of one FP32 block-CSR SpMV launch on this
    workload, from the committed ncu counter summary; None when the kernel's
    sources changed after the counters were taken."""
    try:
        vals = {}
        with open(SPMV_COUNTERS) as f:
            for line in f:
                m = line.strip().strip("`").split(":", 1)
                if len(m) == 2:
                    vals[m[0].strip()] = m[1].strip()
        if vals.get("kernel_sources_sha256") != spmv_source_hash():
            return None
        return float(vals["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


# ----------------------------------------------------------------------------
# algorithmic bytes
# ----------------------------------------------------------------------------

def spmv_bytes(nnzb, bd, n, real_bytes):
    """Bytes one block-CSR SpMV must move: every block value and column index
    once, the source vector once (neighbour reuse from cache) and the output
    once. real_bytes = 4 (FP32) or 8 (FP64)."""
    return nnzb * (bd * bd * 2 * real_bytes + 4) + 2 * n * 2 * real_bytes


def solve_bytes(info, S, nnzb, bd, n, mixed=True):
    """Algorithmic HBM bytes of one solve, from what it ran.

    c = bytes of one complex unknown in the iteration precision (8 mixed,
    16 FP64); "passes" below are reads or writes of one vector.
    Multi-shift iteration k:
      SpMV: every block value and column index once, source and output once;
      r -= alpha Ap with |r|^2: 3 passes;
      update: r, p read + p write (3), every non-base shift still active
      4 passes (3 in its last iteration), the base shift's x 2 passes.
    Mixed only: at every reliable update (the count is reported by the
      library) a fold of each shift's FP32 x into FP64 (x32 read, x64
      read+write = 40 B per unknown; one shift in the refinement stage) and
      one FP64 residual SpMV (+ b read, r write).
    Checks: each check round applies the FP64 operator to every shift it
      checks (round 0: all S; later rounds: the shifts just refined).
    Refinement iteration k: the SpMV reads the matrix once for all refined
      shifts still iterating (they share one launch), plus source and output
      per iterating shift; r update 3 passes and update 5 passes per shift.
    """
    rb = 4 if mixed else 8
    c = 2 * rb
    mat = nnzb * (bd * bd * 2 * rb + 4)
    a_it = mat + 2 * n * c
    a64 = spmv_bytes(nnzb, bd, n, 8) + n * 16 + n * c
    it = int(info.iters)
    conv = np.asarray(info.shift_iters).reshape(-1)
    base = int(np.argmax(conv)) if len(conv) else 0
    total = 0.0
    for k in range(1, it + 1):
        upd = 3 + 2
        for s, cv in enumerate(conv):
            if s == base:
                continue
            cs = cv if cv >= 0 else it
            upd += 4 if k < cs else (3 if k == cs else 0)
        total += a_it + (3 + upd) * n * c
    if mixed:
        # reliable updates of the multi-shift stage (fold every shift) and the
        # final fold of the stage
        ru_main = int(info.reliable_updates) - int(info.refine_reliable_updates)
        total += (ru_main + 1) * S * 40 * n + ru_main * a64
        # refinement-stage updates: fold one shift each
        total += int(info.refine_reliable_updates) * (a64 + 40 * n)
    ref = np.asarray(info.shift_refine_iters).reshape(-1)
    refined = int(np.count_nonzero(ref))
    total += (S + refined * int(info.refine_rounds)) * a64
    kmax = int(ref.max()) if len(ref) else 0
    for k in range(1, kmax + 1):
        act = int(np.count_nonzero(ref >= k))
        total += mat + act * (2 + 3 + 5) * n * c
    return total


def fp64_solve_bytes(info, S, nnzb, bd, n):
    """The plain FP64 form (16 B per complex unknown, x_s updated in place)."""
    return solve_bytes(info, S, nnzb, bd, n, mixed=False)


def multishift_iter_bytes_fp64(S, nnzb, bd, n):
    """FP64 bytes of one CG-M iteration with every shift active (the oracle)."""
    return spmv_bytes(nnzb, bd, n, 8) + (3 + 3 + 4 * (S - 1) + 2) * n * 16


def stencil_solve_bytes(info, S, V, nc, recon, mixed=True):
    """Algorithmic HBM bytes of one solve through the staggered stencil path
    (msc_solve on a staggered operator, nrhs right-hand sides), from what it
    ran. u = bytes of one site's colour vector in the iteration precision
    (8 nc mixed, 16 nc FP64); l = bytes of one site's FP32 links in the four
    directions ((nc-1) nc complex with row reconstruction, else nc^2), l64
    the FP64 links (nc^2 complex). A D pass reads every link once whatever
    the number of right-hand sides it serves (they share the links).
    Multi-shift iteration k (R_k right-hand sides still iterating):
      pass 1 (t = D p, P): links + R_k (p read, t write);
      pass 2 (r -= alpha (d p - D t), |r|^2): links + R_k (t, p, r read, r write);
      update: per right-hand side r, p read + p write, the base shift's x
      read + write, and per non-base shift still iterating x_s, p_s read +
      write (x_s and p_s read + x_s write in its last iteration).
    Mixed only, per reliable update (count reported): fold every shift of
    that right-hand side (x32 read, x64 read + write) and one FP64 residual
    (two FP64 D passes: links64 twice, x64 read, t64 write, t64, x64, b read,
    r write); the stage's final fold of every shift.
    Checks and refinement as in `solve_bytes`, with two FP64 D passes per
    residual and, per refinement iteration, the links once per pass for all
    refined shifts still iterating plus 2 + 4 + 5 vector passes per shift.
    """
    rb = 4 if mixed else 8
    u = 2 * rb * nc
    l = 4 * ((nc - 1) if (mixed and recon) else nc) * nc * 2 * rb
    l64 = 4 * nc * nc * 16
    u64 = 16 * nc
    res64 = 2 * l64 + 2 * u64 + 3 * u64 + u   # one FP64 residual b - (A + s) x, per site
    it_all = np.asarray(info.shift_iters).reshape(-1, S)
    R = it_all.shape[0]
    total = 0.0
    for r in range(R):
        conv = it_all[r]
        base = int(np.argmax(conv))
        itr = int(conv.max())
        for k in range(1, itr + 1):
            upd = 3 + 2
            for s_, cv in enumerate(conv):
                if s_ == base:
                    continue
                upd += 4 if k < cv else (3 if k == cv else 0)
            total += V * (2 * u + 4 * u + upd * u)
    iters = int(info.iters)
    total += iters * 2 * V * l  # links of both passes, shared by the right-hand sides
    if mixed:
        ru_main = int(info.reliable_updates) - int(info.refine_reliable_updates)
        fold = 40 * nc * V
        total += (ru_main + R) * S * fold
        total += ru_main * V * res64
        # refinement-stage updates: one FP64 residual and the fold of one shift
        total += int(info.refine_reliable_updates) * (V * res64 + fold)
    ref = np.asarray(info.shift_refine_iters).reshape(-1)
    refined = int(np.count_nonzero(ref))
    total += (R * S + refined * int(info.refine_rounds)) * V * res64
    kmax = int(ref.max()) if len(ref) else 0
    for k in range(1, kmax + 1):
        act = int(np.count_nonzero(ref >= k))
        total += 2 * V * l + act * V * (2 + 4 + 5) * u
    return total


def stencil_pass_fracs(info, V, nc, recon, nrhs, peak):
    """Live fractions of HBM of the two D passes and the update kernel at the
    sampled multi-shift iterations (every right-hand side iterating):
    algorithmic bytes of one launch / its mean CUDA-event time."""
    u, l = 8 * nc, 4 * ((nc - 1) if recon else nc) * nc * 8
    b1 = V * (l + nrhs * 2 * u)
    b2 = V * (l + nrhs * 4 * u)
    bu = V * u * (5 * nrhs + 4 * float(info.prof_active))
    out = {"pass1_bytes": b1, "pass2_bytes": b2, "update_bytes": bu,
           "pass1_ms": info.op_ms, "pass2_ms": info.rupdate_ms, "update_ms": info.update_ms,
           "update_active_shifts": float(info.prof_active)}
    for k, b, ms in (("pass1", b1, info.op_ms), ("pass2", b2, info.rupdate_ms), ("update", bu, info.update_ms)):
        out[k + "_gbs"] = b / (ms * 1e-3) / 1e9 if ms else None
        out[k + "_frac"] = out[k + "_gbs"] / peak if ms else None
    return out


# ----------------------------------------------------------------------------
# helpers
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(prefix="msc_clocks_", suffix=".csv")
            self.fh = os.fdopen(fd, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.fh,
                stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.fh.close()
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
                for nm, v in zip(names, parts[5:9]):
                    if v.lower() in ("active", "1"):
                        reasons.add(nm)
        try:
            os.remove(self.path)
        except OSError:
            pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax),
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_setup(gpus):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if backend == "nccl":
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
        pg = dist
    return world, rank, local, pg


def barrier(pg, torch):
    if pg is not None:
        if torch.cuda.is_available():
            pg.barrier(device_ids=[torch.cuda.current_device()])
        else:
            pg.barrier()


def reduce_max(pg, torch, v):
    if pg is None:
        return v
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def reduce_sum(pg, torch, v):
    if pg is None:
        return v
    t = torch.tensor([v], dtype=torch.float64,
                     device="cuda" if torch.cuda.is_available() else "cpu")
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


# ----------------------------------------------------------------------------
# CPU oracle (baseline and reference arm)
# ----------------------------------------------------------------------------

def oracle_sample(problem, iters):
    """Time `iters` CG-M iterations of the FP64 oracle on the full workload
    (all 15 shifts active; the oracle applies A in stencil form, the same
    matrix the block-CSR export holds). Returns (seconds, threads)."""
    import oracle
    t = time.perf_counter()
    res = oracle.cgm_staggered(problem.links, problem.dims, problem.nc, problem.mass,
                               problem.b[0], problem.sigma, 0.0, max_iter=iters, freeze=False)
    dt = time.perf_counter() - t
    assert res.iters == iters
    return dt, oracle.num_threads()


def cpu_line(problem, nnzb, bd, n, S, iters, iters_1core=2):
    import oracle
    dt, cores = oracle_sample(problem, iters)
    b = multishift_iter_bytes_fp64(S, nnzb, bd, n) * iters
    out = {"value": b / dt / 1e9, "unit": "GB/s", "cores": cores, "kind": "oracle",
           "ms_per_iteration": 1e3 * dt / iters,
           "sample": f"{iters} CG-M iterations (FP64, all {S} shifts active) of the full "
                     f"24^4 workload, stencil form of the same A"}
    # the same on one host core (the paper's CPU figure is one core)
    oracle.set_threads(1)
    try:
        dt1, _ = oracle_sample(problem, iters_1core)
    finally:
        oracle.set_threads(cores)
    b1 = multishift_iter_bytes_fp64(S, nnzb, bd, n) * iters_1core
    out["one_core"] = {"value": b1 / dt1 / 1e9, "unit": "GB/s", "cores": 1,
                       "ms_per_iteration": 1e3 * dt1 / iters_1core,
                       "sample": f"{iters_1core} CG-M iterations, same workload, one thread"}
    return out


def run_reference(args):
    import torch
    world, rank, local, pg = dist_setup(args.gpus)
    if rank != 0:
        return 0
    from paper_1102_2143_gb300 import inputs
    p = inputs.lattice_24x4_su3_15shifts()
    V = inputs.volume(p.dims)
    n, bd, nnzb, S = V * 3, 3, 33 * V, len(p.sigma)
    iters = 4
    for _ in range(args.warmup):
        oracle_sample(p, 1)
    times = []
    cores = 1
    for _ in range(args.steps):
        dt, cores = oracle_sample(p, iters)
        times.append(dt)
    tot = sum(times)
    b = multishift_iter_bytes_fp64(S, nnzb, bd, n) * iters * args.steps
    val = b / tot / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": val, "unit": "GB/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "form": "FP64 CPU oracle, stencil form of A"},
            "cpu_baseline": {"value": val, "unit": "GB/s", "cores": cores, "kind": "oracle",
                             "sample": f"each step: {iters} CG-M iterations, all {S} shifts"},
            "e2e": {"value": val, "unit": "GB/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------
# the paper's own workload (Sec. 4, Table 1), context beside the headline
# ----------------------------------------------------------------------------

PAPER_T10 = {  # ms per iteration, Table 1 (2-D Poisson, 1000 x 1000, 15 shifts)
    "hardware": "one T10 GPU of an NVIDIA Tesla S1070; CPU: Intel Nehalem 2.67 GHz, one core",
    "cgm_15_shifts_gpu_fp64": 12.9839, "cgm_15_shifts_gpu_fp32": 8.82461,
    "cg_unshifted_gpu_fp64": 3.48276, "cg_unshifted_gpu_fp32": 2.20814,
    "cg_unshifted_cpu_fp64": 159.158,
}


def paper_workload(ctx, msc, inputs, torch, stream):
    """The 1000 x 1000 five-point Poisson operator with 15 shifts through the
    generic block-CSR path (1 x 1 blocks): time to solution and ms per
    multi-shift iteration, FP64 and mixed, and the single unshifted system,
    beside the paper's T10 numbers. Complex arithmetic: the Gaussian source
    is complex, so each iteration carries two real right-hand sides' worth
    of vectors (the matrix is read once)."""
    p = inputs.poisson_2d_15shifts()
    op = msc.msc_op_bsr(ctx, p.n, 1, p.row_ptr, p.col_idx, p.vals)
    b = torch.from_numpy(p.b).cuda()
    out = {"workload": "2-D Poisson five-point, 1000x1000 (10^6 unknowns), Dirichlet; "
                       "15 shifts log-spaced 1e-4..10; complex Gaussian source; tol 1e-10",
           "paper_t10_ms_per_iteration": PAPER_T10}

    def timed(sig, prec):
        x = torch.empty((1, len(sig), p.n), dtype=torch.complex128, device="cuda")
        msc.solve(ctx, op, b, sig, x=x, tol=p.tol, precision=prec)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, info = msc.solve(ctx, op, b, sig, x=x, tol=p.tol, precision=prec)
        e1.record(stream)
        torch.cuda.synchronize()
        assert info.status == 0, info.status
        ms = e0.elapsed_time(e1)
        return {"time_to_solution_ms": ms, "iterations": info.iters,
                "refine_iterations": info.refine_iters,
                "ms_per_iteration": ms / max(1, info.iters + info.refine_iters),
                "max_true_rel_resid": float(np.max(info.true_rel_resid))}

    out["cgm_15_shifts_fp64"] = timed(p.sigma, msc.MSC_FP64)
    out["cgm_15_shifts_mixed"] = timed(p.sigma, msc.MSC_MIXED)
    out["cg_unshifted_fp64"] = timed(np.array([0.0]), msc.MSC_FP64)
    # the paper's comparison: the 15 shifted systems solved one by one
    # (single-shift CG each) against one CG-M solve of all of them
    for prec, name in ((msc.MSC_FP64, "fp64"), (msc.MSC_MIXED, "mixed")):
        sep = [timed(np.array([sg]), prec) for sg in p.sigma]
        tot = sum(r["time_to_solution_ms"] for r in sep)
        out[f"separate_cg_15_shifts_{name}"] = {
            "time_to_solution_ms": tot, "iterations": sum(r["iterations"] for r in sep),
            "max_true_rel_resid": max(r["max_true_rel_resid"] for r in sep),
            "cgm_speedup": tot / out[f"cgm_15_shifts_{name}"]["time_to_solution_ms"]}
    out["cgm_15_fp64_speedup_per_iteration_vs_t10"] = (
        PAPER_T10["cgm_15_shifts_gpu_fp64"] / out["cgm_15_shifts_fp64"]["ms_per_iteration"])
    msc.msc_op_destroy(op)
    return out


# ----------------------------------------------------------------------------
# the other hot-path workloads (secondary measurements beside the headline)
# ----------------------------------------------------------------------------

def stencil_pass_bytes(V, nc, recon):
    """Algorithmic bytes of the two FP32 stencil passes of one iteration (one
    right-hand side): every link once (nc-1 stored rows with reconstruction),
    then pass 1 (t = D p, P fused) reads p and writes t, pass 2 (r -= alpha
    (d p - D t), |r|^2 fused) reads t, p and r and writes r."""
    link = 4 * (nc - 1 if recon else nc) * nc * 8
    vec = nc * 8
    return V * (link + 2 * vec), V * (link + 4 * vec)


LARGEST = ("32^4 SU(3) staggered A=M^dag M (stencil, two-row FP32 links), m=0.01, eps=0.9, "
           "20 shifts 1e-5..10, 8 Gaussian RHS, mixed FP32/FP64, reliable updates every 50 "
           "iterations at the latest, tol 1e-10 FP64 true residual per shift")


def largest_config(ctx, msc, inputs, torch, stream, steps=2, fp64=True):
    """The largest workload that fits one GPU, measured like the headline:
    time to solution of all 160 shifted systems, algorithmic GB/s of the
    whole solve, the live fractions of the two D passes and the update
    kernel, end to end through the C ABI with host buffers, and the plain
    FP64 form of the same solve."""
    peak, peak_kind = load_peaks()
    p = inputs.lattice_32x4_su3_20shifts()
    V, S, R = inputs.volume(p.dims), len(p.sigma), p.b.shape[0]
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    recon = msc.msc_op_recon(op)
    b = torch.from_numpy(p.b).cuda()
    x = torch.empty((R, S, p.n), dtype=torch.complex128, device="cuda")

    def run(bb, xx, prec=msc.MSC_MIXED):
        _, info = msc.solve(ctx, op, bb, p.sigma, x=xx, tol=p.tol, precision=prec)
        assert info.status == 0, info.status
        return info

    run(b, x)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    infos = [run(b, x) for _ in range(steps)]
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    info = infos[-1]
    nbytes = stencil_solve_bytes(info, S, V, p.nc, recon)
    fr = stencil_pass_fracs(info, V, p.nc, recon, R, peak)
    out = {"workload": LARGEST, "steps": steps, "time_to_solution_ms": ms,
           "value": nbytes / (ms * 1e-3) / 1e9, "unit": "GB/s", "frac_of_peak": nbytes / (ms * 1e-3) / 1e9 / peak,
           "algorithmic_bytes": nbytes, "iterations": info.iters, "refine_iterations": info.refine_iters,
           "refine_system_iterations": int(np.sum(info.shift_refine_iters)),
           "reliable_updates": info.reliable_updates,
           "iters_per_s": (info.iters + info.refine_iters) / (ms * 1e-3),
           "max_true_rel_resid": float(np.max(info.true_rel_resid)), "gpu_launches": info.kernel_launches,
           "kernels_live": fr, "peak": peak, "peak_source": peak_kind,
           "timing": "CUDA events on the solve's stream; pass and update times sampled inside the solve's graphs"}
    roof = []
    for k, kern in (("pass1", "k_stag_group PASS_A (t = D p, P fused; links once per group of right-hand sides)"),
                    ("pass2", "k_stag_group PASS_B (r -= alpha (d p - D t), |r|^2 fused)"),
                    ("update", "k_update (fused multi-shift update)")):
        if fr[k + "_gbs"]:
            roof.append({"kernel": kern, "bound": "hbm", "achieved": fr[k + "_gbs"], "peak": peak, "unit": "GB/s",
                         "frac": fr[k + "_frac"], "bytes_per_launch": fr[k + "_bytes"], "launch_ms": fr[k + "_ms"]})
    out["roofline"] = roof
    # end to end: pinned host source and solution
    bh = torch.from_numpy(p.b).pin_memory()
    xh = torch.empty((R, S, p.n), dtype=torch.complex128).pin_memory()
    torch.cuda.synchronize()
    e0.record(stream)
    ie = run(bh, xh)
    e1.record(stream)
    torch.cuda.synchronize()
    ms_e = e0.elapsed_time(e1)
    out["e2e"] = {"value": stencil_solve_bytes(ie, S, V, p.nc, recon) / (ms_e * 1e-3) / 1e9, "unit": "GB/s",
                  "ms_per_step": ms_e, "h2d_bytes_per_step": R * p.n * 16, "d2h_bytes_per_step": R * S * p.n * 16}
    del xh, bh
    if fp64:
        torch.cuda.synchronize()
        e0.record(stream)
        i64 = run(b, x, msc.MSC_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        out["fp64_plain"] = {"time_to_solution_ms": ms64, "iterations": i64.iters,
                             "value": stencil_solve_bytes(i64, S, V, p.nc, recon, mixed=False) / (ms64 * 1e-3) / 1e9,
                             "unit": "GB/s", "pass1_fp64_ms": i64.op_ms, "pass2_fp64_ms": i64.rupdate_ms,
                             "max_true_rel_resid": float(np.max(i64.true_rel_resid))}
        out["speedup_vs_fp64_plain"] = ms64 / ms
    # the same source restricted to even sites through the single-parity solve
    # against the full-lattice solve of the embedded source (one right-hand side)
    msc.msc_op_destroy(op)
    del x, b
    return out


def parity_workload(ctx, msc, inputs, torch, stream):
    """A source on the even sites of the 32^4 lattice (20 shifts, 1 RHS): the
    single-parity solve on half the unknowns against msc_solve on the
    embedded full-lattice source."""
    p = inputs.lattice_32x4_su3_20shifts(nrhs=1)
    V, S = inputs.volume(p.dims), len(p.sigma)
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    x = np.arange(V)
    c = [x % p.dims[0], (x // p.dims[0]) % p.dims[1], (x // (p.dims[0] * p.dims[1])) % p.dims[2],
         x // (p.dims[0] * p.dims[1] * p.dims[2])]
    even = np.nonzero(((c[0] + c[1] + c[2] + c[3]) & 1) == 0)[0]
    bh = p.b[0].reshape(V, p.nc)[even].reshape(-1)
    bf = np.zeros((V, p.nc), dtype=np.complex128)
    bf[even] = bh.reshape(-1, p.nc)
    bh_d = torch.from_numpy(bh).cuda()
    bf_d = torch.from_numpy(bf.reshape(-1)).cuda()
    out = {"workload": "32^4 SU(3), m=0.01, eps=0.9, 20 shifts 1e-5..10, one Gaussian source on the even "
                       "sites, mixed, tol 1e-10"}
    for name, fn in (("full_lattice", lambda: msc.solve(ctx, op, bf_d, p.sigma, tol=p.tol)),
                     ("single_parity", lambda: msc.solve_parity(ctx, op, 0, bh_d, p.sigma, tol=p.tol))):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, info = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        assert info.status == 0, info.status
        out[name] = {"time_to_solution_ms": e0.elapsed_time(e1), "iterations": info.iters,
                     "refine_iterations": info.refine_iters, "pass1_ms": info.op_ms, "pass2_ms": info.rupdate_ms,
                     "update_ms": info.update_ms, "max_true_rel_resid": float(np.max(info.true_rel_resid))}
    out["speedup"] = out["full_lattice"]["time_to_solution_ms"] / out["single_parity"]["time_to_solution_ms"]
    msc.msc_op_destroy(op)
    return out


def poly_rhs_workload(ctx, msc, inputs, torch, stream):
    """Different right-hand side per shift, b_s = q_s(A) b with quadratic q_s
    (16^4 SU(3), 20 shifts, mixed): msc_solve_poly_rhs (one CG-M sequence
    after polynomial division) against forming each b_s with the FP64
    operator and solving the 20 shifted systems one by one."""
    p = inputs.lattice_32x4_su3_20shifts(L=16, nrhs=1)
    S = len(p.sigma)
    coef = inputs.rng(9100).uniform(-1.0, 1.0, size=(S, 3))
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    b = torch.from_numpy(p.b[0]).cuda()
    x = torch.empty((S, p.n), dtype=torch.complex128, device="cuda")
    tmp = torch.empty_like(b)

    def poly_solve():
        return msc.solve_poly_rhs(ctx, op, b, p.sigma, coef, x=x, tol=p.tol)

    def one_by_one():
        infos = []
        for s in range(S):
            bs = coef[s, 2] * b
            msc.msc_op_apply(ctx, op, 0.0, bs, tmp, msc.MSC_FP64)
            bs = tmp + coef[s, 1] * b
            msc.msc_op_apply(ctx, op, 0.0, bs, tmp, msc.MSC_FP64)
            bs = tmp + coef[s, 0] * b
            _, info = msc.solve(ctx, op, bs, p.sigma[s:s + 1], x=x[s:s + 1][None], tol=p.tol)
            infos.append(info)
        return None, infos

    out = {"workload": "16^4 SU(3), m=0.01, eps=0.9, 20 shifts 1e-5..10, b_s = q_s(A) b with q_s quadratic "
                       "(coefficients uniform in [-1, 1]), mixed, tol 1e-10 relative to |b_s|"}
    for name, fn in (("poly_rhs_cgm", poly_solve), ("one_by_one", one_by_one)):
        fn()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        _, info = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        out[name] = {"time_to_solution_ms": e0.elapsed_time(e1)}
        if name == "poly_rhs_cgm":
            out[name].update({"iterations": info.iters, "refine_iterations": info.refine_iters,
                              "max_true_rel_resid": float(np.max(info.true_rel_resid))})
        else:
            out[name].update({"iterations": int(sum(i.iters + i.refine_iters for i in info)),
                              "max_true_rel_resid": float(max(np.max(i.true_rel_resid) for i in info))})
    out["speedup"] = out["one_by_one"]["time_to_solution_ms"] / out["poly_rhs_cgm"]["time_to_solution_ms"]
    msc.msc_op_destroy(op)
    return out


def other_workloads(ctx, msc, inputs, torch, stream):
    out = {}
    peak, _ = load_peaks()

    def ev_time(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        r = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1), r

    # the small correctness workload: 4^4 SU(3), 8 shifts, FP64 and mixed
    # (latency-bound; time to solution, median of 5 after a warm-up)
    p = inputs.lattice_4x4_su3_8shifts()
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    b = torch.from_numpy(p.b).cuda()
    small = {"workload": "4^4 SU(3) staggered, m=0.1, eps=0.5, 8 shifts 1e-3..1, 1 RHS, tol 1e-10 "
                         "(768 complex unknowns; latency-bound)"}
    for prec, name in ((msc.MSC_FP64, "fp64"), (msc.MSC_MIXED, "mixed")):
        msc.solve(ctx, op, b, p.sigma, tol=p.tol, precision=prec)
        ts = []
        for _ in range(5):
            ms_, (_, info) = ev_time(lambda: msc.solve(ctx, op, b, p.sigma, tol=p.tol, precision=prec))
            ts.append(ms_)
        small[name] = {"time_to_solution_ms": float(np.median(ts)), "iterations": info.iters,
                       "refine_iterations": info.refine_iters, "max_true_rel_resid": float(np.max(info.true_rel_resid))}
    out["lattice_4x4_su3_8shifts"] = small
    msc.msc_op_destroy(op)

    # staggered stencil path: 32^4 SU(3), m = 0.01, eps = 0.9, 20 shifts, 1 RHS
    p = inputs.lattice_32x4_su3_20shifts(nrhs=1)
    V = inputs.volume(p.dims)
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    recon = msc.msc_op_recon(op)
    b = torch.from_numpy(p.b).cuda()
    x = torch.empty((1, len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
    msc.solve(ctx, op, b, p.sigma, x=x, tol=p.tol)
    ms, (_, info) = ev_time(lambda: msc.solve(ctx, op, b, p.sigma, x=x, tol=p.tol))
    assert info.status == 0, info.status
    b1, b2 = stencil_pass_bytes(V, p.nc, recon)
    out["stencil_32x4_20shifts_mixed"] = {
        "workload": "32^4 SU(3) staggered A=M^dag M (stencil, two-row FP32 links), m=0.01, eps=0.9, "
                    "20 shifts 1e-5..10, 1 RHS, mixed, tol 1e-10",
        "time_to_solution_ms": ms, "iterations": info.iters, "refine_iterations": info.refine_iters,
        "max_true_rel_resid": float(np.max(info.true_rel_resid)),
        "pass1_ms": info.op_ms, "pass2_ms": info.rupdate_ms, "update_ms": info.update_ms,
        "pass1_gbs": b1 / (info.op_ms * 1e-3) / 1e9, "pass2_gbs": b2 / (info.rupdate_ms * 1e-3) / 1e9,
        "pass1_frac": b1 / (info.op_ms * 1e-3) / 1e9 / peak,
        "pass2_frac": b2 / (info.rupdate_ms * 1e-3) / 1e9 / peak,
        "pass_bytes": [b1, b2], "timing": "pass times: CUDA events around the pass nodes inside the solve's graphs"}
    msc.msc_op_destroy(op)
    del x, b

    # batched uneven systems: 64 problems in one batch against one by one
    probs = inputs.batched_uneven_systems(64)
    ops = [msc.msc_op_staggered(ctx, q.nc, q.dims, torch.from_numpy(q.links).cuda(), q.mass)
           for q in probs]
    items = [(o, torch.from_numpy(q.b).cuda(), q.sigma) for o, q in zip(ops, probs)]
    msc.solve_batched(ctx, items)
    ms_b, (_, infos, tun) = ev_time(lambda: msc.solve_batched(ctx, items))
    ms_s, _ = ev_time(lambda: [msc.solve(ctx, o, bb, sg) for o, bb, sg in items])
    assert all(i.status == 0 for i in infos)
    bbytes = sum(stencil_solve_bytes(i, len(q.sigma), inputs.volume(q.dims), q.nc, msc.msc_op_recon(o))
                 for i, q, o in zip(infos, probs, ops))
    out["batched_64_uneven_mixed"] = {
        "workload": "64 staggered problems, L in {4..12}, SU(2)/SU(3), m in [0.02,0.2], eps=0.6, "
                    "4..20 shifts 1e-4..1, 4 RHS each, mixed, tol 1e-10",
        "batched_ms": ms_b, "one_by_one_ms": ms_s, "speedup": ms_s / ms_b,
        "algorithmic_bytes": bbytes, "batched_gbs": bbytes / (ms_b * 1e-3) / 1e9,
        "batched_over_hbm_copy": bbytes / (ms_b * 1e-3) / 1e9 / peak,
        "one_by_one_gbs": bbytes / (ms_s * 1e-3) / 1e9,
        "bytes": "sum over the 64 problems of the stencil solve's algorithmic bytes (bench.stencil_solve_bytes); "
                 "the systems are small (at most 12^4 sites, vectors of at most 0.5 MB), so their working "
                 "sets stay in the 129 MB L2 and the rate can exceed the HBM copy bandwidth",
        "tuned_shape": {"site_threads": tun.site_threads, "vec_threads": tun.vec_threads,
                        "vec_units": tun.vec_units}}
    for o in ops:
        msc.msc_op_destroy(o)

    # non-Hermitian family: the staggered Dirac multi-mass solve
    # (m + sigma_s + D) x_s = b by BiCGStab-M (FP64, block-CSR, 9 blocks per
    # row), beside CG-M (mixed) on the normal equations of the same family
    # (A = m0^2 - D^2, shifts m_s^2 - m0^2; x_s would then need one more D)
    dims, nc, m0 = (24, 24, 24, 24), 3, 0.05
    U = inputs.su_n_links(dims, nc, 0.6, 6000)
    rp, ci, va = inputs.staggered_dirac_bsr(U, dims, nc, m0)
    Vd = inputs.volume(dims)
    sig = inputs.log_shifts(1e-3, 1.0, 12)
    bd = torch.from_numpy(inputs.gaussian_source(Vd * nc, 6001)).cuda()
    dop = msc.msc_op_bsr(ctx, Vd, nc, rp, ci, va)
    xd = torch.empty((1, len(sig), Vd * nc), dtype=torch.complex128, device="cuda")
    msc.solve_nonherm(ctx, dop, bd, sig, x=xd)
    ms_b, (_, info_b) = ev_time(lambda: msc.solve_nonherm(ctx, dop, bd, sig, x=xd))
    assert info_b.status == 0, info_b.status
    msc.msc_op_destroy(dop)
    sop = msc.msc_op_staggered(ctx, nc, dims, torch.from_numpy(U).cuda(), m0 + sig[0])
    nsig = (m0 + sig) ** 2 - (m0 + sig[0]) ** 2
    msc.solve(ctx, sop, bd, nsig, x=xd)
    ms_c, (_, info_c) = ev_time(lambda: msc.solve(ctx, sop, bd, nsig, x=xd))
    msc.msc_op_destroy(sop)
    out["dirac_multimass_24x4_bicgstabm"] = {
        "workload": "24^4 SU(3) staggered Dirac M = m + D (m=0.05, eps=0.6) as block-CSR, 12 masses "
                    "m + sigma_s, sigma_s log-spaced 1e-3..1, 1 RHS, tol 1e-10",
        "bicgstabm_fp64_ms": ms_b, "bicgstabm_iterations": info_b.iters,
        "bicgstabm_ms_per_iteration": ms_b / max(1, info_b.iters),
        "max_true_rel_resid": float(np.max(info_b.true_rel_resid)),
        "cgm_normal_equations_mixed_ms": ms_c, "cgm_normal_iterations": info_c.iters,
        "note": "BiCGStab-M: two FP64 block-CSR applications per iteration (FP64-ALU bound on GB300); "
                "the CG-M route solves (m_s^2 - D^2) y_s = b and needs x_s = (m_s - D) y_s after"}
    del xd

    # adjoint: 16^4 SU(3), 12 (sigma_s, c_s); solve, S and dS/dphi, dS/dU
    p, c = inputs.lattice_16x4_su3_force()
    op = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    phi = torch.from_numpy(p.b[0]).cuda()
    x = torch.empty((1, len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
    dphi = torch.empty(p.n, dtype=torch.complex128, device="cuda")
    dU = torch.empty(p.links.shape, dtype=torch.complex128, device="cuda")
    msc.solve(ctx, op, phi, p.sigma, x=x, tol=p.tol)
    ms_solve, _ = ev_time(lambda: msc.solve(ctx, op, phi, p.sigma, x=x, tol=p.tol))
    ms_grad, _ = ev_time(lambda: msc.msc_quad_form_grad(ctx, op, len(p.sigma), c, x[0], dphi, dU))
    out["adjoint_16x4_12shifts"] = {
        "workload": "16^4 SU(3), m=0.05, eps=0.7, 12 shifts 1e-4..5, c_s = sigma_s^0.5/12; "
                    "S = sum c_s phi^dag (A+sigma_s)^-1 phi",
        "solve_ms": ms_solve, "grad_ms": ms_grad,
        "grad": "dS/dphi and the link force dS/dU from the solved x_s (FP64 D x_s passes + outer products)"}
    msc.msc_op_destroy(op)
    return out


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-aux", action="store_true",
                    help="skip the secondary workloads (stencil 32^4, batched, adjoint)")
    ap.add_argument("--no-paper", action="store_true",
                    help="skip the paper's own 2-D Poisson workload (context numbers)")
    ap.add_argument("--fp64-steps", type=int, default=3)
    ap.add_argument("--no-largest", action="store_true",
                    help="skip the largest single-GPU workload (32^4, 8 RHS, 20 shifts)")
    ap.add_argument("--largest-steps", type=int, default=2)
    ap.add_argument("--no-fp64-largest", action="store_true",
                    help="skip the plain FP64 form of the largest workload")
    ap.add_argument("--profile-region", action="store_true",
                    help="bracket the device-timed steps with cudaProfilerStart/Stop "
                         "(for ncu --profile-from-start off)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1102_2143_gb300 as msc
    from paper_1102_2143_gb300 import inputs

    world, rank, local, pg = dist_setup(args.gpus)
    torch.cuda.set_device(local)
    stream = torch.cuda.current_stream()
    msc.load()

    p = inputs.lattice_24x4_su3_15shifts()
    V = inputs.volume(p.dims)
    S = len(p.sigma)
    ctx = msc.msc_create(local, stream)
    sop = msc.msc_op_staggered(ctx, p.nc, p.dims, torch.from_numpy(p.links).cuda(), p.mass)
    nbr, nnzb, bd = msc.msc_op_bsr_size(sop)
    rp = torch.empty(nbr + 1, dtype=torch.int64, device="cuda")
    ci = torch.empty(nnzb, dtype=torch.int32, device="cuda")
    va = torch.empty((nnzb, bd, bd), dtype=torch.complex128, device="cuda")
    msc.msc_staggered_export_bsr(ctx, sop, rp, ci, va)
    op = msc.msc_op_bsr(ctx, nbr, bd, rp, ci, va)
    del va, rp, ci
    msc.msc_op_destroy(sop)
    n = nbr * bd
    b_dev = torch.from_numpy(p.b[0]).cuda()
    x_dev = torch.empty((1, S, n), dtype=torch.complex128, device="cuda")
    b_host = torch.from_numpy(p.b[0]).pin_memory()
    x_host = torch.empty((1, S, n), dtype=torch.complex128).pin_memory()

    def step(b, x, precision=msc.MSC_MIXED):
        x, info = msc.solve(ctx, op, b, p.sigma, x=x, tol=p.tol, precision=precision)
        assert info.status == 0, info.status
        return info

    for _ in range(max(args.warmup, 3)):
        step(b_dev, x_dev)
    torch.cuda.synchronize()

    # ---- timed region: device-resident inputs --------------------------------
    clocks = ClockSampler(torch.cuda.current_device())
    clocks.start()
    barrier(pg, torch)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    infos = []
    if args.profile_region:
        torch.cuda.profiler.start()
    ev0.record(stream)
    for _ in range(args.steps):
        infos.append(step(b_dev, x_dev))
    ev1.record(stream)
    torch.cuda.synchronize()
    if args.profile_region:
        torch.cuda.profiler.stop()
    barrier(pg, torch)
    clk = clocks.stop()
    ms_local = ev0.elapsed_time(ev1) / args.steps
    ms = reduce_max(pg, torch, ms_local)
    bytes_local = sum(solve_bytes(i, S, nnzb, bd, n) for i in infos) / args.steps
    bytes_all = reduce_sum(pg, torch, bytes_local)
    value = bytes_all / (ms * 1e-3) / 1e9
    launches = sum(i.kernel_launches for i in infos)

    # roofline of the dominant kernel (FP32 block-CSR SpMV), sampled live
    op_ms = [i.op_ms for i in infos if i.prof_samples > 0]
    spmv_ms = float(np.mean(op_ms)) if op_ms else None
    spmv_b = spmv_bytes(nnzb, bd, n, 4)
    peak, peak_kind = load_peaks()
    roof = None
    if spmv_ms:
        ach = spmv_b / (spmv_ms * 1e-3) / 1e9
        # the fused multi-shift update at the same sampled iterations: r, p
        # read, p write, the base shift's x read + write, and x_s, p_s read +
        # write for every non-base shift still iterating (count sampled live)
        upd_ms = float(np.mean([i.update_ms for i in infos]))
        upd_act = float(np.mean([i.prof_active for i in infos]))
        upd_b = (5 + 4 * upd_act) * n * 8
        roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                "traffic": load_spmv_traffic(), "kernel": "k_bsr_a1<3> (FP32 SpMV + fused P)",
                "bytes_per_launch": spmv_b, "launch_ms": spmv_ms, "peak_source": peak_kind,
                "update_kernel_ms": upd_ms, "update_active_shifts": upd_act, "update_bytes_per_launch": upd_b,
                "update_frac": upd_b / (upd_ms * 1e-3) / 1e9 / peak if upd_ms else None,
                "rupdate_kernel_ms": float(np.mean([i.rupdate_ms for i in infos])),
                "rupdate_frac": 3 * n * 8 / (float(np.mean([i.rupdate_ms for i in infos])) * 1e-3) / 1e9 / peak}

    # ---- end to end: host source and solution buffers ------------------------
    barrier(pg, torch)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    einfos = []
    for _ in range(args.steps):
        einfos.append(step(b_host, x_host))
    e1.record(stream)
    torch.cuda.synchronize()
    barrier(pg, torch)
    e2e_ms = reduce_max(pg, torch, e0.elapsed_time(e1) / args.steps)
    e2e_bytes = reduce_sum(pg, torch, sum(solve_bytes(i, S, nnzb, bd, n) for i in einfos) / args.steps)
    e2e = {"value": e2e_bytes / (e2e_ms * 1e-3) / 1e9, "unit": "GB/s", "ms_per_step": e2e_ms,
           "h2d_bytes_per_step": n * 16, "d2h_bytes_per_step": S * n * 16}

    # ---- plain FP64 form of the same solve -----------------------------------
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    step(b_dev, x_dev, msc.MSC_FP64)
    torch.cuda.synchronize()
    f0.record(stream)
    finfos = [step(b_dev, x_dev, msc.MSC_FP64) for _ in range(args.fp64_steps)]
    f1.record(stream)
    torch.cuda.synchronize()
    f_ms = f0.elapsed_time(f1) / args.fp64_steps
    fp64 = {"time_to_solution_ms": f_ms, "iterations": finfos[-1].iters,
            "value": fp64_solve_bytes(finfos[-1], S, nnzb, bd, n) / (f_ms * 1e-3) / 1e9,
            "unit": "GB/s", "spmv_fp64_launch_ms": finfos[-1].op_ms}

    # the paper's comparison on the headline workload: the 15 shifted systems
    # solved one at a time (single-shift mixed solves of the same matrix)
    separate = None
    if rank == 0 and not args.no_aux:
        msc.solve(ctx, op, b_dev, p.sigma[:1], x=x_dev[:, :1], tol=p.tol)  # warm-up (graphs)
        torch.cuda.synchronize()
        s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s0.record(stream)
        sinfo = []
        for sg in p.sigma:
            _, i1 = msc.solve(ctx, op, b_dev, np.array([sg]), x=x_dev[:, :1], tol=p.tol)
            sinfo.append(i1)
        s1.record(stream)
        torch.cuda.synchronize()
        sep_ms = s0.elapsed_time(s1)
        separate = {"time_to_solution_ms": sep_ms, "iterations": int(sum(i.iters + i.refine_iters for i in sinfo)),
                    "max_true_rel_resid": float(max(np.max(i.true_rel_resid) for i in sinfo)),
                    "cgm_speedup": sep_ms / ms,
                    "what": "each of the 15 shifts solved on its own (mixed, same matrix and tolerance)"}

    aux = None
    if rank == 0 and not args.no_aux:
        aux = other_workloads(ctx, msc, inputs, torch, stream)
        aux["single_parity_32x4_20shifts"] = parity_workload(ctx, msc, inputs, torch, stream)
        aux["poly_rhs_16x4_20shifts"] = poly_rhs_workload(ctx, msc, inputs, torch, stream)

    largest = None
    if rank == 0 and not args.no_largest:
        largest = largest_config(ctx, msc, inputs, torch, stream, steps=args.largest_steps,
                                 fp64=not args.no_fp64_largest)

    paper = None
    if rank == 0 and not args.no_paper:
        paper = paper_workload(ctx, msc, inputs, torch, stream)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_line(p, nnzb, bd, n, S, iters=6)

    if rank == 0:
        last = infos[-1]
        line = {
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world,
            "steps": args.steps, "warmup": max(args.warmup, 3), "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "lattice": list(p.dims), "nc": 3, "block_rows": nbr,
                       "blocks": nnzb, "shifts": S, "rhs": 1, "tol": p.tol, "mass": p.mass,
                       "eps": p.eps, "reliable_every": 50,
                       "l2": "inputs larger than L2 (FP32 blocks %.0f MB, FP64 blocks %.0f MB)"
                             % (nnzb * 76 / 1e6, nnzb * 148 / 1e6),
                       "parallelism": f"replicas x{world}"},
            "time_to_solution_ms": ms, "iterations": last.iters,
            "refine_iterations": last.refine_iters, "refine_rounds": last.refine_rounds,
            "iters_per_s": (last.iters + last.refine_iters) / (ms * 1e-3),
            "max_true_rel_resid": float(np.max(last.true_rel_resid)),
            "fp64_plain": fp64, "speedup_vs_fp64_plain": f_ms / ms, "separate_single_shift": separate,
            "e2e": e2e, "gpu_launches": launches, "roofline": roof, "cpu_baseline": cpu,
            "paper_workload": paper, "other_workloads": aux, "largest_config": largest,
            "clocks": clk,
        }
        print(json.dumps(line), flush=True)
    msc.msc_op_destroy(op)
    msc.msc_destroy(ctx)
    if pg is not None:
        # the other ranks wait for rank 0's secondary workloads, then all
        # leave together
        barrier(pg, torch)
        pg.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
