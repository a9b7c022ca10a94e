"""Benchmark of the shifted Green's-function path on GB300.

One step = one gb_shifted_solve over the whole workload: every (shift, RHS)
pair of the 50-monomer PPV-like chain (N = 1900 orbitals, 128 shifts on
[-15, 10] eV + 0.02i, all 1900 unit right-hand sides), mixed precision,
tol 1e-6, reduced to LDOS / density / energy-density / charge / energy.

Prints one JSON line (rank 0).  --impl reference times the CPU oracle (dense
LU per shift) on a bounded sample of the same workload instead.
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

METRIC = "RHS·shift solves/s at rel err ≤1e-6 vs plain FP64 GPU; SpMM HBM GB/s % of peak"
UNIT = "RHS·shift solves/s"
NOMINAL_MAX_SM_MHZ = 2070.0
# DRAM bytes (read + write) per launch from ncu captures of the current
# kernels, for roofline.traffic; None once a kernel changes, until it is
# captured again.  spmm_quad_kernel<1> (FP32, one column) on the block-aligned
# bundle Hamiltonian:
SPMM_F32_W1_DRAM_BYTES = 271.619584e6
# team_kernel<mixed> with the exact factor inner solve on the 1900-orbital
# chain, bytes per column-iteration of a 60-iteration capture (84.54 GB over
# 114,000 column-iterations), scaled to a launch by its column-iterations:
TEAM_MIXED_DRAM_BYTES_PER_COL_ITER = 741.6e3


def spmm_alg_bytes(info, v, W):
    """Algorithmic bytes of one sparse product with W complex columns: values
    of the true nonzeros, block indices and row pointers, read X, write Y."""
    return v * info["nnz"] + 4 * info["nnzb"] + 4 * (info["nb"] + 1) + 2 * (2 * v) * info["n"] * W


def team_alg_bytes_per_col_iter(info, W, K, mean_row, inner_per_outer, method, v=4):
    """Algorithmic bytes the shifted COCG must move per column-iteration.

    Per outer iteration of a W-column panel: the H p product; the inner solve
    (iterative: n_in x (S product + 5 vector passes); exact factor: per level
    the triangular blocks D^-1, D^-T and the band blocks E, F plus 8 vector
    passes (read f, write / read t, y, u, write x), and one S product for the
    float-float residual between the two mixed levels); the seed update (10
    vector passes); the per-shift projected state 4 x 16 B x |R_j| x K read and
    written plus the 16 B x |R_j| gather of r.  Divided by W.
    """
    N = info["n"]
    vec = 2 * v * N * W  # one pass over a complex panel vector
    b = spmm_alg_bytes(info, v, W)
    if method == "factor":
        nblk, bw = info["factor_nblk"], info["factor_bw"]
        factor = v * (2 * nblk * 2080 + 2 * nblk * 64 * bw)
        levels = inner_per_outer
        b += levels * (factor + 8 * vec) + (levels - 1) * spmm_alg_bytes(info, v, W)
    else:
        b += inner_per_outer * (spmm_alg_bytes(info, v, W) + 5 * vec)
    b += 10 * vec
    b += W * (4 * 16 * mean_row * K + 16 * mean_row)
    return b / W


def dense_peaks(torch):
    """FP64 and FP32 (no TF32) dense GEMM throughput of this GPU, TFLOP/s,
    measured live with cuBLAS: the ALU roofs of the FP64 and FP32 paths."""
    out = {}
    for name, dt, n in (("fp64", torch.float64, 4096), ("fp32", torch.float32, 8192)):
        prev = torch.backends.cuda.matmul.allow_tf32
        torch.backends.cuda.matmul.allow_tf32 = False
        a = torch.randn(n, n, dtype=dt, device="cuda")
        b = torch.randn(n, n, dtype=dt, device="cuda")
        c = a @ b
        torch.cuda.synchronize()
        best = 1e30
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            c = a @ b
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        torch.backends.cuda.matmul.allow_tf32 = prev
        out[name] = 2.0 * n**3 / (best / 1e3) / 1e12
        del a, b, c
    return out


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="ppv1900")
    ap.add_argument("--panel", type=int, default=0, help="RHS per panel (0: library choice)")
    ap.add_argument("--no-check", action="store_true", help="skip the FP64-GPU accuracy check")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-fp64", action="store_true", help="skip the plain-FP64 GPU comparison run")
    ap.add_argument("--no-chain800", action="store_true", help="skip the 800-orbital FP64 chain line")
    ap.add_argument("--no-spmm", action="store_true", help="skip the bundle-scale SpMM bandwidth measurement")
    ap.add_argument("--spmm-only", type=str, default="",
                    help="comma-separated panel widths: only the bundle SpMM bandwidth measurement")
    ap.add_argument("--batched", action="store_true",
                    help="uneven-chain batch (512 chains, sampled RHS) in one persistent launch")
    ap.add_argument("--bundle", action="store_true",
                    help="bundle-scale solve throughput, mixed versus plain FP64 (short runs)")
    ap.add_argument("--surrogate", action="store_true",
                    help="measure the learned surrogate with solver judge instead of the solver step")
    ap.add_argument("--fermi", action="store_true",
                    help="ppv1900: chemical potential, Fermi-weighted rho / P^E and atomic forces from one solve")
    ap.add_argument("--wavepacket", action="store_true",
                    help="ppv1900 wavepacket propagation (32 packets, 100 steps of 0.1 fs)")
    ap.add_argument("--poles", action="store_true",
                    help="ppv1900 density matrices from a 40-pole expansion of the Fermi function")
    ap.add_argument("--maxit", type=int, default=0, help="override the workload's iteration cap")
    ap.add_argument("--flags", type=int, default=0,
                    help="gb_solve_params.flags for the timed solve (4: CG, 16: Chebyshev inner iteration)")
    ap.add_argument("--profile-case", action="store_true",
                    help="run one solve of the workload (for ncu captures) and exit")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        try:
            with open(path) as f:
                return json.load(f), "measured"
        except Exception:
            pass
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def max_over_ranks(x: float, device) -> float:
    """The largest x over all ranks of the initialised process group (x itself
    without one): replicas are timed by the slowest rank."""
    import torch
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    t = torch.tensor([float(x)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------- clocks
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join(os.environ.get("GB_CLOCK_LOG_DIR", "/tmp"), f"gbgreen_clocks_{gpu_index}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
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
        self.f.close()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------- our arm
def run_ours(args):
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import workload

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl")
    wl = workload(args.workload)
    system, z, cols = wl["system"], wl["z"], wl["cols"]
    K, nrhs = len(z), len(cols)
    mat = gbg.Matrix(system)
    info = mat.info
    kw = dict(tol=wl["tol"], maxit=args.maxit or wl["maxit"], prec=wl["prec"], w_rho=wl["w_rho"],
              w_edm=wl["w_edm"], panel=args.panel, inner_tol=wl.get("inner_tol", 0.0), flags=args.flags)
    plan = gbg.solve_plan(mat, z, cols, tol=wl["tol"], maxit=wl["maxit"], prec=wl["prec"], panel=args.panel,
                          flags=args.flags)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    def step(ws=None):
        return gbg.shifted_solve(mat, z, cols, workspace=ws, **kw)

    out = step()
    ws = out["workspace"]
    for _ in range(max(args.warmup - 1, 0)):
        out = step(ws)
    assert out["status"] == 0, out["message"]
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    if world > 1:
        torch.distributed.barrier()
    clocks.start()
    times = []
    for _ in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = step(ws)
        e1.record(stream)
        torch.cuda.synchronize()
        times.append(e0.elapsed_time(e1))
    clk = clocks.stop()
    total_ms = max_over_ranks(float(sum(times)), "cuda")
    ms_per_step = total_ms / args.steps
    solves = K * nrhs
    value = world * solves * args.steps / (total_ms / 1e3)
    iters = out["iters"].cpu().numpy().astype(np.int64)
    inner = out["inner_iters"].cpu().numpy().astype(np.int64)
    W = plan["panel"]
    npan = (nrhs + W - 1) // W
    it_p = np.array([iters[p * W : (p + 1) * W].max() for p in range(npan)])
    inner_per_outer = float(inner[::W].sum() / max((it_p + 1).sum(), 1))
    method = "factor" if plan["inner"] == "factor" else "iterative"
    mean_row = float(np.mean(np.diff(system.row_ptr)[cols]))
    bpc = team_alg_bytes_per_col_iter(info, W, K, mean_row, round(inner_per_outer) if method == "factor"
                                      else inner_per_outer, method, v=4 if wl["prec"] == "mixed" else 8)
    col_iters = float(iters.sum())
    alg_bytes = bpc * col_iters  # per launch = per step
    achieved_gbs = alg_bytes / (ms_per_step / 1e3) / 1e9
    peaks, peak_src = measured_peaks()
    hbm_peak = float(peaks.get("hbm_gbs", 6800.0))
    res = {
        "metric": METRIC,
        "value": value,
        "unit": UNIT,
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_per_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32x2+f32 (f64 scalars)" if wl["prec"] == "mixed" else "f64",
        "data": "synthetic",
        "config": {
            "workload": "ppv1900: 50-monomer PPV-like chain, N=1900 orbitals (38/monomer), 128 shifts on "
                        "[-15,10] eV + 0.02i, all 1900 RHS e_j, mixed precision, tol 1e-6",
            "rhs": nrhs, "shifts": K, "n": int(system.n), "panel": W, "teams": plan["teams"],
            "inner_solve": plan["inner"], "flags": args.flags,
            "l2": "256 MB flush between timed steps (workspace also exceeds L2)",
            "parallelism": "replicas" if world > 1 else "1 GPU",
        },
        "krylov_iters_per_s": col_iters * world * args.steps / (total_ms / 1e3),
        "outer_iters": {"min": int(iters.min()), "median": int(np.median(iters)), "max": int(iters.max())},
        "inner_per_outer": inner_per_outer,
        "gpu_launches": args.steps,
        "roofline": {
            "kernel": "team_kernel<mixed>" if wl["prec"] == "mixed" else "team_kernel<fp64>",
            "bound": "hbm",
            "achieved": achieved_gbs,
            "peak": hbm_peak,
            "unit": "GB/s",
            "frac": achieved_gbs / hbm_peak,
            "traffic": TEAM_MIXED_DRAM_BYTES_PER_COL_ITER * col_iters
            if (TEAM_MIXED_DRAM_BYTES_PER_COL_ITER and wl["prec"] == "mixed" and args.workload == "ppv1900"
                and method == "factor") else None,
            "peak_source": f"{peak_src}: MEASURED_PEAKS hbm_gbs" if peak_src == "measured" else "fallback 6.8 TB/s",
            "alg_bytes_per_col_iter": bpc,
            "col_iters_per_launch": col_iters,
            "model": "algorithmic bytes per column-iteration (H p product, inner solve, seed update, per-shift "
                     "projected state; v = 4 B mixed / 8 B FP64, true nonzeros) x column-iterations / step time; "
                     "the panel vectors partly hit L2, so this HBM fraction is L2-assisted",
        },
        "clocks": clk,
    }
    # accuracy against the plain FP64 GPU path on sampled columns (outside the timed region)
    if not args.no_check and rank == 0:
        rng = np.random.default_rng(0)
        sidx = np.sort(rng.choice(nrhs, size=16, replace=False))
        # reference: the plain FP64 path converged well past the workload tolerance
        ref = gbg.shifted_solve(mat, z, cols[sidx], tol=1e-10, maxit=30000, prec="fp64",
                                w_rho=wl["w_rho"], w_edm=wl["w_edm"], panel=1)
        off = out["off"]
        errs = {}
        for key in ("ldos", "q", "e_loc"):
            a = out[key].cpu().numpy()
            a = a[:, sidx] if a.ndim == 2 else a[sidx]
            b = ref[key].cpu().numpy()
            errs[key] = float(np.abs(a - b).max() / np.abs(b).max())
        for key in ("rho", "edm"):
            a = out[key].cpu().numpy()
            a = np.concatenate([a[off[j] : off[j + 1]] for j in sidx])
            b = ref[key].cpu().numpy()
            errs[key] = float(np.abs(a - b).max() / np.abs(b).max())
        res["rel_err_vs_fp64_gpu"] = errs
        res["rel_err_max"] = max(errs.values())
        # FP64 true residual of the same 16 columns as this solve produces them
        rt = gbg.true_residual(mat, z, cols, sidx, tol=wl["tol"], maxit=args.maxit or wl["maxit"], prec=wl["prec"],
                               inner_tol=wl.get("inner_tol", 0.0), panel=args.panel, flags=args.flags)
        est = out["resid"].cpu().numpy()[:, sidx]
        res["true_residual_check"] = {"columns": 16, "pairs": int(rt.numel()),
                                      "true_max": float(rt.max().item()), "estimate_max": float(est.max()),
                                      "pairs_above_tol": int((rt > wl["tol"]).sum().item()),
                                      "note": "||e_j - (z_k S - H) x^k||_2 in FP64 from the full-history re-run "
                                              "(gb_true_residual) vs the recursive estimate"}
    # the plain FP64 GPU solver on the same workload and tolerance: one launch,
    # outside the timed region (both paths then meet rel err <= 1e-6)
    if not args.no_fp64 and rank == 0 and wl["prec"] == "mixed":
        p64 = gbg.solve_plan(mat, z, cols, tol=wl["tol"], maxit=wl["maxit"], prec="fp64")
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f64 = gbg.shifted_solve(mat, z, cols, tol=wl["tol"], maxit=args.maxit or wl["maxit"], prec="fp64",
                                w_rho=wl["w_rho"], w_edm=wl["w_edm"])
        e1.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        it64 = f64["iters"].cpu().numpy()
        res["fp64_gpu"] = {"value": solves / (ms64 / 1e3), "unit": UNIT, "seconds": ms64 / 1e3,
                           "status": int(f64["status"]), "tol": wl["tol"], "panel": p64["panel"],
                           "inner_solve": p64["inner"], "krylov_iters_per_s": float(it64.sum()) / (ms64 / 1e3),
                           "outer_iters_max": int(it64.max()),
                           "workload": "same pairs, shifts, weights and tol as the timed mixed step"}
        res["mixed_over_fp64"] = value / res["fp64_gpu"]["value"]
        del f64
    # configs' plain-FP64 case: the 800-orbital chain, every pair, one launch
    if not args.no_chain800 and rank == 0 and args.workload == "ppv1900":
        res["chain800_fp64"] = run_chain800(gbg, torch)
    # end to end through the public API with host buffers
    if not args.no_e2e:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2 = gbg.Matrix(system)  # host CSR -> device inside gb_build_bsr
        del ws
        out = None
        o2 = gbg.shifted_solve(m2, z, cols, **kw)  # allocates its workspace (torch caching allocator)
        host = {k: o2[k].cpu() for k in ("ldos", "rho", "edm", "q", "e_loc", "iters", "converged", "resid")}
        torch.cuda.synchronize()
        e2e_s = time.perf_counter() - t0
        m2.close()
        h2d = (system.row_ptr.nbytes + system.col_idx.nbytes + system.h_val.nbytes + system.s_val.nbytes
               + K * 16 * 3 + nrhs * 4)
        d2h = sum(v.numel() * v.element_size() for v in host.values())
        res["e2e"] = {"value": world * solves / e2e_s, "unit": UNIT, "h2d_bytes_per_step": int(h2d),
                      "d2h_bytes_per_step": int(d2h),
                      "includes": "host CSR upload and factor build (gb_build_bsr), workspace allocation, "
                                  "the solve, device-to-host copy of every output"}
    # SpMM bandwidth on the bundle-scale Hamiltonian (the metric's second part)
    if not args.no_spmm and rank == 0:
        res["spmm_hbm"] = measure_spmm(gbg, torch)
    # CPU oracle on a bounded sample (rank 0 at N = 1 only)
    if not args.no_cpu and rank == 0 and world == 1:
        res["cpu_baseline"] = cpu_oracle_rate(wl, n_shift=8)
    mat.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    if rank == 0:
        print(json.dumps(res), flush=True)


def run_chain800(gbg, torch):
    """Plain FP64 solve of the 800-orbital 4-orbital chain: 64 shifts on
    [-12, 12] eV + 0.05i, all 800 unit right-hand sides, tol 1e-10 (maxit
    8000: the stated 800 iterations do not converge the mid-band shifts)."""
    from synth import workload

    wl = workload("chain800")
    m0 = gbg.Matrix(wl["system"])
    kw = dict(tol=wl["tol"], maxit=8000, prec="fp64", w_rho=wl["w_rho"], w_edm=wl["w_edm"])
    r = gbg.shifted_solve(m0, wl["z"], wl["cols"], **kw)  # warm-up
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    r = gbg.shifted_solve(m0, wl["z"], wl["cols"], workspace=r["workspace"], **kw)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    it = r["iters"].cpu().numpy()
    plan = gbg.solve_plan(m0, wl["z"], wl["cols"], tol=wl["tol"], maxit=8000, prec="fp64")
    pairs = len(wl["z"]) * len(wl["cols"])
    out = {"value": pairs / (ms / 1e3), "unit": UNIT, "seconds": ms / 1e3, "status": int(r["status"]),
           "converged_all": bool(r["converged"].cpu().numpy().all()), "panel": plan["panel"],
           "inner_solve": plan["inner"], "outer_iters_max": int(it.max()),
           "krylov_iters_per_s": float(it.sum()) / (ms / 1e3),
           "workload": "chain800: 200 sites x 4 orbitals, 64 shifts on [-12,12] eV + 0.05i, all 800 RHS, FP64, "
                       "tol 1e-10, maxit 8000"}
    m0.close()
    return out


# ---------------------------------------------------------------- SpMM bandwidth
def measure_spmm(gbg, torch, widths=(1, 2, 4, 8, 16, 32, 64), reps=10):
    """gb_spmm (Y = H X) on the condensed-bundle Hamiltonian (N = 321,100).

    Algorithmic bytes per launch: v*nnz (values) + 4*nnzb (block columns)
    + 4*(nb+1) (block row pointers) + 2*(2v)*N*W (read X, write Y), v = 4
    (FP32) or 8 (FP64) -- true nonzeros only, so the 4x4 padding of the
    block format counts against the kernel.  X and Y exceed L2 at these sizes
    only together with the matrix (>= 300 MB per launch), so every launch
    streams from HBM.
    """
    from synth import workload

    system = workload("bundle169")["system"]
    mat = gbg.Matrix(system)
    info = mat.info
    n, nnz, nnzb, nb = info["n"], info["nnz"], info["nnzb"], info["nb"]
    peaks, src = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    alu = dense_peaks(torch)  # TFLOP/s, measured live (cuBLAS DGEMM / SGEMM without TF32)
    stream = torch.cuda.current_stream()
    rows = []
    for prec, v in (("fp32", 4), ("fp64", 8)):
        for w in widths:
            if prec == "fp64" and w > 8:
                continue  # FP64 is FMA-bound at every width; wider panels only scale the time
            dt = torch.complex64 if prec == "fp32" else torch.complex128
            x = torch.randn(n, w, dtype=dt, device="cuda")
            y = torch.empty_like(x)
            for _ in range(3):
                mat.spmm(0, x, prec=prec, out=y)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            # a ~2.5 ms spin ahead of the timed launches lets the host queue all
            # of them, so the events see back-to-back kernels, not Python gaps
            torch.cuda._sleep(5_000_000)
            e0.record(stream)
            for _ in range(reps):
                mat.spmm(0, x, prec=prec, out=y)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            alg = v * nnz + 4 * nnzb + 4 * (nb + 1) + 2 * (2 * v) * n * w
            stored = v * 16 * nnzb + 4 * nnzb + 4 * (nb + 1) + 2 * (2 * v) * n * w
            flops = 4.0 * nnz * w
            flops_padded = 4.0 * 16 * nnzb * w  # executed: every stored 4x4 entry, 2 FMA per complex column
            hbm_ms = alg / (peak * 1e9) * 1e3
            alu_ms = flops_padded / (alu[prec] * 1e12) * 1e3
            bound = "hbm" if hbm_ms >= alu_ms else "alu"
            rows.append({"prec": prec, "w": w, "ms": ms, "algorithmic_bytes": int(alg), "stored_bytes": int(stored),
                         "achieved_gbs": alg / (ms / 1e3) / 1e9, "stored_gbs": stored / (ms / 1e3) / 1e9,
                         "useful_tflops": flops / (ms / 1e3) / 1e12, "executed_tflops": flops_padded / (ms / 1e3) / 1e12,
                         "hbm_floor_ms": hbm_ms, "alu_floor_ms": alu_ms, "binding_roof": bound,
                         "frac_of_binding_roof": max(hbm_ms, alu_ms) / ms})
            del x, y
    mat.close()
    best = max((r for r in rows if r["prec"] == "fp32"), key=lambda r: r["achieved_gbs"])
    return {
        "kernel": "spmm_kernel (gb_spmm, Y = H X)",
        "workload": f"bundle169 H: N={n}, nnz={nnz}, 4x4 blocks nnzb={nnzb} (fill {nnz / (16 * nnzb):.3f})",
        "bound": "hbm",
        "achieved": best["achieved_gbs"], "peak": peak, "unit": "GB/s", "frac": best["achieved_gbs"] / peak,
        "peak_source": src, "best": {"prec": best["prec"], "w": best["w"]}, "sweep": rows,
        "alu_peaks_tflops": alu,
        "alu_note": "FP64 / FP32 roofs: cuBLAS DGEMM / SGEMM (no TF32) measured in this run; the FP64 product is "
                    "ALU-bound on GB300 (its FMA floor exceeds the HBM floor)",
        "traffic": SPMM_F32_W1_DRAM_BYTES if (best["prec"], best["w"]) == ("fp32", 1) else None,
    }


# ---------------------------------------------------------------- oracle (CPU)
def cpu_oracle_rate(wl, n_shift: int):
    import oracle

    system, z = wl["system"], wl["z"]
    idx = np.linspace(0, len(z) - 1, n_shift).round().astype(int)
    zs = z[idx]
    cols = wl["cols"]
    t0 = time.perf_counter()
    oracle.solve_outputs(system, zs, cols, wl["w_rho"][idx], wl["w_edm"][idx])
    dt = time.perf_counter() - t0
    return {"value": len(zs) * len(cols) / dt, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{len(zs)} of {len(z)} shifts x all {len(cols)} RHS (dense complex LU per shift, "
                      f"NumPy/SciPy FP64), {dt:.1f} s"}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from synth import workload

    wl = workload(args.workload)
    n_shift = 2
    for _ in range(args.warmup):
        cpu_oracle_rate(wl, n_shift)
    rates = []
    t0 = time.perf_counter()
    for _ in range(args.steps):
        rates.append(cpu_oracle_rate(wl, n_shift))
    total = time.perf_counter() - t0
    solves = n_shift * len(wl["cols"]) * args.steps
    value = solves / total
    res = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        "config": {"workload": "ppv1900 (bounded sample: 2 shifts x all 1900 RHS per step)"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                         "sample": rates[-1]["sample"]},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(res), flush=True)


def run_surrogate(args):
    """Surrogate (q, E) outputs/s with the solver as judge vs the plain solver.

    Labels: the batched mixed solver on 24 seeded 2x2-chain x 6-monomer bundles
    (912 orbitals each, 48 shifts on [-15, 10] eV + 0.2i, tol 1e-6).  Inference:
    a fresh 3x3 x 10-monomer bundle (3,420 orbitals): descriptors, MLP, 5%
    random re-solve plus out-of-range fallback, versus solving every orbital.
    """
    import torch

    import paper_1603_09616_gb300 as gbg
    from paper_1603_09616_gb300 import surrogate as sg
    from synth import fermi_weights, ppv_bundle, shift_grid

    torch.cuda.set_device(0)
    z = shift_grid(-15.0, 10.0, 48, 0.2)
    w_rho, w_edm = fermi_weights(z)
    train = [ppv_bundle(n_side=2, n_mono=6, seed=1000 + s) for s in range(24)]
    mats = [gbg.Matrix(s) for s in train]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    labels = sg.solve_local_outputs(mats, train, z, w_rho, w_edm, tol=1e-6, maxit=6000)
    torch.cuda.synchronize()
    t_labels = time.perf_counter() - t0
    X = torch.cat([sg.descriptors(m, s) for m, s in zip(mats, train)])
    Y = torch.cat([torch.stack([q.float(), e.float()], dim=1) for q, e in labels]).contiguous()
    sur = sg.Surrogate(seed=0)
    t0 = time.perf_counter()
    hist = sur.fit(X, Y, epochs=80, batch=1024, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    fresh = ppv_bundle(n_side=3, n_mono=10, seed=4242)
    mf = gbg.Matrix(fresh)
    cols = np.arange(fresh.n, dtype=np.int32)
    gbg.shifted_solve(mf, z, cols[:64], tol=1e-6, maxit=6000, prec="mixed", w_rho=w_rho, w_edm=w_edm)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    full = gbg.shifted_solve(mf, z, cols, tol=1e-6, maxit=6000, prec="mixed", w_rho=w_rho, w_edm=w_edm)
    torch.cuda.synchronize()
    t_plain = time.perf_counter() - t0
    q, e, rep = sg.infer_with_judge(sur, mf, fresh, z, w_rho, w_edm, tol=1e-6, maxit=6000, sample_frac=0.05,
                                    threshold=1e-3)
    qf, ef = full["q"].cpu().numpy(), full["e_loc"].cpu().numpy()
    pred = sur.predict(sg.descriptors(mf, fresh)).cpu().numpy()
    qn, en = q.cpu().numpy(), e.cpu().numpy()
    res = {
        "metric": "surrogate local outputs (q_j, E_j) per second with the shifted solver as judge",
        "value": fresh.n / rep["t_total_s"], "unit": "orbitals/s", "n_gpus": 1, "higher_is_better": True,
        "plain_solver": {"value": fresh.n / t_plain, "unit": "orbitals/s", "seconds": t_plain},
        "speedup_vs_plain": t_plain / rep["t_total_s"],
        "network_mae": {"q": float(np.abs(pred[:, 0] - qf).mean()), "E": float(np.abs(pred[:, 1] - ef).mean())},
        "mean_predictor_mae": {"q": float(np.abs(Y[:, 0].mean().item() - qf).mean()),
                               "E": float(np.abs(Y[:, 1].mean().item() - ef).mean())},
        "judged_output_mae": {"q": float(np.abs(qn - qf).mean()), "E": float(np.abs(en - ef).mean())},
        "judged_output_max_err": {"q": float(np.abs(qn - qf).max()), "E": float(np.abs(en - ef).max())},
        "judge": rep, "train": {"samples": int(X.shape[0]), "label_seconds": t_labels, "train_seconds": t_train,
                                "loss_first": hist[0], "loss_last": hist[-1]},
        "config": {"workload": "surrogate: train 24 x (2x2 chains x 6 monomers, 912 orbitals), infer 3x3 x 10 "
                               "(3420 orbitals); 48 shifts on [-15,10] eV + 0.2i; judge 5% + out-of-range"},
        "dtype": "bf16 weights, f32 accumulation", "data": "synthetic",
    }
    print(json.dumps(res), flush=True)


def run_bundle(args):
    """Bundle-scale (N = 321,100) solve throughput, mixed and plain FP64.

    Short solves (maxit outer iterations, 64 shifts on [-15, 10] eV + 0.02i)
    measure the outer-iteration rate without waiting for convergence: mixed on
    2048 of the configuration's 4096 random columns (8-column panels; the
    workspace holds ten N-long float-float vectors per column, ~51 MB, so all
    4096 at once would need ~210 GB), and mixed and FP64 on the same 256
    columns for the precision ratio.  Reported: Krylov column-iterations per
    second of each.
    """
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import workload

    torch.cuda.set_device(0)
    wl = workload("bundle169")
    mat = gbg.Matrix(wl["system"])
    maxit = args.maxit or 10
    out = {}
    for tag, prec, ncol in (("mixed_2048", "mixed", 2048), ("mixed_256", "mixed", 256), ("fp64_256", "fp64", 256)):
        cols = wl["cols"][:ncol]
        gbg.shifted_solve(mat, wl["z"], cols[:8], tol=1e-12, maxit=2, prec=prec, raise_on=(-1, -2, -3, -4))
        torch.cuda.synchronize()
        plan = gbg.solve_plan(mat, wl["z"], cols, tol=1e-12, maxit=maxit, prec=prec)
        t0 = time.perf_counter()
        r = gbg.shifted_solve(mat, wl["z"], cols, tol=1e-12, maxit=maxit, prec=prec, w_rho=wl["w_rho"],
                              w_edm=wl["w_edm"], raise_on=(-1, -2, -3, -4))
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        it = r["iters"].cpu().numpy()
        out[tag] = {"columns": ncol, "panel": plan["panel"], "teams": plan["teams"], "seconds": dt,
                    "outer_iterations": int(it.max()), "column_iterations_per_s": float(it.sum()) / dt,
                    "inner_per_outer": float(r["inner_iters"].cpu().numpy().sum() / max(it.sum(), 1))}
        del r
    res = {"metric": "bundle-scale shifted-COCG column-iterations/s (mixed; mixed vs plain FP64)",
           "value": out["mixed_2048"]["column_iterations_per_s"], "unit": "column-iterations/s", "n_gpus": 1,
           "higher_is_better": True, "cases": out,
           "mixed_over_fp64_same_columns": out["mixed_256"]["column_iterations_per_s"]
           / out["fp64_256"]["column_iterations_per_s"],
           "config": {"workload": f"bundle169: N={wl['system'].n}, nnz={wl['system'].nnz}, 64 shifts on "
                                  f"[-15,10] eV + 0.02i, {maxit} outer iterations (throughput, not convergence)"},
           "data": "synthetic"}
    print(json.dumps(res), flush=True)


def run_batched(args):
    """Uneven-chain batch: 512 chains (76..1900 orbitals, 32..256 shifts each,
    eta 0.02, tol 1e-6), 8 sampled unit right-hand sides per chain, in one
    gb_shifted_solve_batched launch whose panel width the library's autotuner
    picks from {8, 16, 32} (probe runs of 40 iterations, outside the timed
    region), followed by the FP64 correction solve of any column that misses
    tol.  Timed: the launch plus the correction (CUDA events; the correction's
    share is reported as correct_ms).  Chains numbered by align_blocks.  Then the same
    batch in plain FP64 for the ratio.  Solves/s = sum over chains of shifts x
    right-hand sides / time."""
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import uneven_batch

    torch.cuda.set_device(0)
    systems, problems = uneven_batch(eta=0.02, cols_per_chain=8, align=True)
    mats = [gbg.Matrix(s) for s in systems]
    stream = torch.cuda.current_stream()
    _, tinfo = gbg.shifted_solve_batched(mats, problems, prec="mixed", tune_probe_maxit=40)
    panel = tinfo["tuned_panel"]
    pairs = sum(len(p["z"]) * len(p["cols"]) for p in problems)
    n = np.array([s.n for s in systems])
    out = {}
    for prec in ("mixed", "fp64"):
        steps = args.steps if prec == "mixed" else 1
        for _ in range(max(args.warmup, 1) if prec == "mixed" else 0):
            res, info = gbg.shifted_solve_batched(mats, problems, prec=prec, panel=panel, correct=True)
            assert info["status"] == 0, info["message"]
        torch.cuda.synchronize()
        times = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            res, info = gbg.shifted_solve_batched(mats, problems, prec=prec, panel=panel, correct=True)
            e1.record(stream)
            torch.cuda.synchronize()
            times.append(e0.elapsed_time(e1))
        assert info["status"] == 0, info["message"]
        ms = sum(times) / len(times)
        iters = np.concatenate([r["iters"].cpu().numpy() for r in res])
        out[prec] = {"value": pairs / (ms / 1e3), "ms": ms, "corrected_columns": info.get("corrected", 0),
                     "correct_ms": info.get("correct_ms", 0.0),
                     "krylov_iters_per_s": float(iters.sum()) / (ms / 1e3),
                     "outer_iters": {"min": int(iters.min()), "median": int(np.median(iters)),
                                     "max": int(iters.max())}}
    m = out["mixed"]
    print(json.dumps({
        "metric": "uneven-chain batch RHS·shift solves/s (one persistent launch + correction)", "value": m["value"],
        "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms"],
        "higher_is_better": True, "dtype": "f32x2+f32 (f64 scalars)", "data": "synthetic",
        "config": {"workload": f"512 PPV-like chains, N {n.min()}..{n.max()} (mean {n.mean():.0f}), "
                               f"32..256 shifts each on [-15,10] eV + 0.02i, 8 sampled RHS per chain, tol 1e-6, "
                               f"autotuned panel {panel}, FP64 correction of columns that miss tol",
                   "pairs": int(pairs), "panel": panel, "tune_times_ms": tinfo["tune_times_ms"]},
        "mixed": m, "fp64": out["fp64"], "mixed_over_fp64": m["value"] / out["fp64"]["value"],
    }), flush=True)
    for mm in mats:
        mm.close()


def run_poles(args):
    """ppv1900's density and energy-density matrices at finite temperature
    (mu = 0, kT = 0.1 eV, the real-axis rule's values) from a 40-pole expansion
    of the Fermi function: 40 shifts at Im z >= pi kT instead of 128 at
    eta = 0.02, all 1900 columns, mixed, then the S^-1 terms
    (gb_add_sinv_terms).  Timed with CUDA events: solve + S^-1 terms.  Error
    against the exact finite-temperature matrices from the host
    eigen-decomposition (the real-axis rule converges to a broadened
    approximation of them instead)."""
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import pole_weights, workload

    torch.cuda.set_device(0)
    wl = workload("ppv1900")
    system = wl["system"]
    cols = wl["cols"]
    z, c, ce, a_r, b_e, c_s = pole_weights(mu=0.0, kT=0.1, n_poles=40)
    mat = gbg.Matrix(system)
    stream = torch.cuda.current_stream()
    lines = {}
    for tol in (1e-6, 1e-8):
        for _ in range(max(args.warmup, 1)):
            out = gbg.shifted_solve(mat, z, cols, tol=tol, maxit=16000, prec="mixed", w_rho=c, w_edm=ce)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        out = gbg.shifted_solve(mat, z, cols, tol=tol, maxit=16000, prec="mixed", w_rho=c, w_edm=ce)
        gbg.add_sinv_terms(mat, cols, out, a_r, b_e, c_s)
        e1.record(stream)
        torch.cuda.synchronize()
        assert out["status"] == 0, out["message"]
        its = out["iters"].cpu().numpy()
        lines[tol] = dict(ms=e0.elapsed_time(e1), outer_iters_max=int(its.max()), outer_iters_median=int(np.median(its)),
                          rho=out["rho"].cpu().numpy(), edm=out["edm"].cpu().numpy())
    import scipy.linalg as sla

    H, S = system.dense()
    lam, Y = sla.eigh(H, S)
    f = 0.5 * (1.0 - np.tanh(lam / 0.2))
    rho_e = 2.0 * (Y * f) @ Y.T
    edm_e = 2.0 * (Y * (f * lam)) @ Y.T
    rows = np.repeat(np.arange(system.n), np.diff(system.row_ptr))
    # packed order: column j's pattern rows (the CSR row j, by symmetry)
    ref_rho, ref_edm = rho_e[system.col_idx, rows], edm_e[system.col_idx, rows]
    res = {"metric": "ppv1900 density matrix from a 40-pole Fermi expansion (seconds, all 1900 columns)",
           "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "cases": {}}
    for tol, d in lines.items():
        err = max(np.abs(d["rho"] - ref_rho).max() / np.abs(ref_rho).max(),
                  np.abs(d["edm"] - ref_edm).max() / np.abs(ref_edm).max())
        res["cases"][f"tol_{tol:g}"] = {"seconds": d["ms"] / 1e3, "shifts": len(z),
                                        "outer_iters_max": d["outer_iters_max"],
                                        "outer_iters_median": d["outer_iters_median"],
                                        "rel_err_vs_eigen": float(err)}
    res["value"] = res["cases"]["tol_1e-08"]["seconds"]
    res["note"] = ("real-axis rule for the same columns: 128 shifts at eta 0.02, up to ~12,000 outer iterations, "
                   "a broadened (eta) approximation of these matrices")
    print(json.dumps(res), flush=True)
    mat.close()


def run_fermi(args):
    """ppv1900 (mixed, real-axis grid, all 1900 columns, G kept): the chemical
    potential for one electron per orbital and the Fermi-weighted rho / P^E
    (gb_fermi_density), then the atomic forces from them (gb_forces), each
    timed with CUDA events after the solve."""
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import model_gradients, workload

    torch.cuda.set_device(0)
    wl = workload("ppv1900")
    system, z, cols = wl["system"], wl["z"], wl["cols"]
    mat = gbg.Matrix(system)
    t0 = time.perf_counter()
    out = gbg.shifted_solve(mat, z, cols, tol=wl["tol"], maxit=wl["maxit"], prec="mixed",
                            inner_tol=wl.get("inner_tol", 0.0), want_g=True)
    torch.cuda.synchronize()
    t_solve = time.perf_counter() - t0
    assert out["status"] == 0, out["message"]
    gh, gs = model_gradients(system)
    atom_off = np.concatenate([[0], np.cumsum(system.atom_norb)]).astype(np.int64)
    stream = torch.cuda.current_stream()
    res = {}
    for rep in range(2):
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        fd = gbg.fermi_density(mat, z, cols, out, float(system.n), 0.1)
        e1.record(stream)
        F = gbg.forces(mat, cols, fd["rho"], fd["edm"], gh, gs, atom_off)
        e2.record(stream)
        torch.cuda.synchronize()
        res = {"fermi_density_ms": e0.elapsed_time(e1), "forces_ms": e1.elapsed_time(e2)}
    Fh = F.cpu().numpy()
    print(json.dumps({"metric": "ppv1900 chemical potential + Fermi-weighted rho/P^E and forces after one solve",
                      "value": res["fermi_density_ms"] + res["forces_ms"], "unit": "ms", "higher_is_better": False,
                      "n_gpus": 1, "data": "synthetic", **res, "solve_s": t_solve, "mu": fd["mu"],
                      "electron_count": float(fd["q"].sum().item()), "atoms": int(len(Fh)),
                      "force_sum_over_max": float(np.abs(Fh.sum(axis=0)).max() / np.abs(Fh).max()),
                      "note": "includes the host-side bisection over the 128 total-DOS values and the transposed "
                              "pattern positions built on the host for the force traces"}), flush=True)
    mat.close()


def run_wavepacket(args):
    """Wavepacket propagation on ppv1900: 32 packets (the HOMO and 31 seeded
    random states) by 100 steps of 0.1 fs (gb_wavepacket, Chebyshev series of
    exp(-i tau S^-1 H), FP64).  Timed with CUDA events; checked against the
    host spectral sum (eigen-decomposition) at the end."""
    import scipy.linalg as sla
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import workload

    torch.cuda.set_device(0)
    system = workload("ppv1900")["system"]
    H, S = system.dense()
    lam, Y = sla.eigh(H, S)
    span = lam.max() - lam.min()
    e_min, e_max = lam.min() - 0.01 * span, lam.max() + 0.01 * span
    rng = np.random.default_rng(5)
    c0 = rng.standard_normal((system.n, 32)) + 1j * rng.standard_normal((system.n, 32))
    c0[:, 0] = Y[:, system.n // 2 - 1]  # the HOMO at one electron per orbital
    tau, steps = 0.1 / 0.6582119569, 100
    mat = gbg.Matrix(system)
    stream = torch.cuda.current_stream()
    psi = torch.from_numpy(np.ascontiguousarray(c0)).cuda()
    gbg.wavepacket(mat, psi.clone(), 2, tau, e_min, e_max)  # warm-up
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    psi, nterms = gbg.wavepacket(mat, psi, steps, tau, e_min, e_max)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    ref = Y @ (np.exp(-1j * lam * steps * tau)[:, None] * (Y.T @ (S @ c0)))
    got = psi.cpu().numpy()
    err = float(np.abs(got - ref).max() / np.abs(ref).max())
    print(json.dumps({"metric": "ppv1900 wavepacket steps x packets per second (0.1 fs steps)",
                      "value": steps * 32 / (ms / 1e3), "unit": "packet-steps/s", "higher_is_better": True,
                      "n_gpus": 1, "data": "synthetic", "ms": ms, "steps": steps, "packets": 32,
                      "terms_per_step": nterms, "rel_err_vs_spectral_sum": err,
                      "simulated_fs_per_s": steps * 0.1 / (ms / 1e3)}), flush=True)
    mat.close()


def run_profile_case(args):
    """One gb_shifted_solve of the workload (short with --maxit), for ncu."""
    import torch

    import paper_1603_09616_gb300 as gbg
    from synth import workload

    torch.cuda.set_device(0)
    wl = workload(args.workload)
    mat = gbg.Matrix(wl["system"])
    out = gbg.shifted_solve(mat, wl["z"], wl["cols"], tol=wl["tol"], maxit=args.maxit or wl["maxit"],
                            prec=wl["prec"], w_rho=wl["w_rho"], w_edm=wl["w_edm"], panel=args.panel,
                            inner_tol=wl.get("inner_tol", 0.0), raise_on=(-1, -2, -3, -4))
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.workload, "status": out["status"],
                      "plan": gbg.solve_plan(mat, wl["z"], wl["cols"], prec=wl["prec"], panel=args.panel)}))


if __name__ == "__main__":
    a = parse()
    if a.spmm_only:
        import torch

        import paper_1603_09616_gb300 as gbg

        torch.cuda.set_device(0)
        print(json.dumps(measure_spmm(gbg, torch, widths=tuple(int(w) for w in a.spmm_only.split(",")))))
    elif a.profile_case:
        run_profile_case(a)
    elif a.fermi:
        run_fermi(a)
    elif a.wavepacket:
        run_wavepacket(a)
    elif a.poles:
        run_poles(a)
    elif a.surrogate:
        run_surrogate(a)
    elif a.bundle:
        run_bundle(a)
    elif a.batched:
        run_batched(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
