"""Benchmark of the GIPC Gauss-Newton hot path on GB300.

One step = one pass of the whole hot path over the C1 batch workload:
  1. eps_x and per-stencil barrier energy, gradient and PSD-projected Hessian for
     1,000,000 contact stencils (40% PT, 30% EE, 10% PE, 10% PP, 6/2/2% nearly
     parallel EE/PE/PP; distances log-uniform in [1e-4 dhat, dhat]),
  2. assembly of the gradient and of the 3x3-block BSR Hessian (mass + blocks) over a
     301,088-vertex two-sheet index space (~4.1M blocks), pattern by key sort,
  3. 200 iterations of block-Jacobi modified PCG (tolerance 0, so all run).
The metric counts stencils per second through the whole step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gipc|reference]
                  [--precision fp64|mixed] [--hess-mode dense|rank1]

Under torchrun (N > 1) every rank runs its own independent batch (weak scaling,
no data-path collective); the step time is the max over ranks.
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "stencil grad+PSD-Hessian/s & Newton iters/s, FP64 vs mixed at ≤1e-4 rel err"
K_STENCILS = 1_000_000
PCG_ITERS = 200
KAPPA = 1e3
HBM_PEAK_FALLBACK = 6800.0        # GB/s, recipe fallback
FP64_PEAK = 152 * 4 * 2.070       # GFLOP/s: 152 SMs x 2 FP64 FMA/clk x 2070 MHz (nominal 1.25 TFLOP/s)
FP32_PEAK = 152 * 256 * 2.070     # GFLOP/s: 152 SMs x 128 FP32 FMA/clk x 2070 MHz
PROF_EVERY = 8                     # per-iteration solver kernels: one CUDA-event span per 8 launches


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gipc", choices=["gipc", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    ap.add_argument("--hess-mode", default="dense", choices=["dense", "rank1"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--product", default="native", choices=["native", "float_pair"],
                    help="arithmetic of the solver's H c for FP64 matrices (the headline uses native)")
    ap.add_argument("--newton-steps", type=int, default=4,
                    help="implicit time steps of the sphere-grid scene per precision (0: skip)")
    ap.add_argument("--batch-steps", type=int, default=3,
                    help="time steps of the 256-scene batch, batched and one scene at a time (0: skip)")
    ap.add_argument("--diff-steps", type=int, default=10,
                    help="checkpointed steps of the beam-on-plate scene differentiated by the adjoint (0: skip)")
    ap.add_argument("--c2-steps", type=int, default=3,
                    help="time steps of the per-step FP64 / mixed converged-position comparison (0: skip)")
    ap.add_argument("--per-type", type=int, default=0, metavar="K",
                    help="instead of the step: evaluate K stencils of each type alone, FP64 and mixed, "
                         "3x3 sub-block output, and print the rate per type (K-stencil launches)")
    return ap.parse_args()


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return HBM_PEAK_FALLBACK, "fallback"


# ----------------------------------------------------------------------------- ranks
def rank_env():
    """(world, rank, local rank) from the torchrun environment (1, 0, 0 without it)."""
    return (int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")),
            int(os.environ.get("LOCAL_RANK", "0")))


def max_over_ranks(value, world, device):
    """The largest of every rank's value (the job's time is that of its slowest rank)."""
    if world <= 1:
        return float(value)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank, world, ms):
    """Whole-job throughput: every rank processes its own batch of units_per_rank in (at most) ms."""
    return units_per_rank * world / (ms * 1e-3)


def workload(seed_offset=0):
    import synth
    d = synth.batch_stencils(K_STENCILS, seed=20230810 + seed_offset)
    st_sheet, n, ids = synth.sheet_index_space(K_STENCILS, seed=20230811 + seed_offset, return_ids=True)
    return {"x": d["x"], "st_own": d["stencils"], "dhat": d["dhat"], "st_sheet": st_sheet, "n": n,
            "mass": synth.sheet_mass(), "sheet_ids": ids}


def workload_desc(args):
    return (f"C1 batch: {K_STENCILS} stencils (own-vertex geometry, 3.7M vertex slots) -> "
            f"{args.hess_mode} {'FP64' if args.precision == 'fp64' else 'FP32'} Hessian blocks"
            f"{' (stored as element-major 3x3 sub-blocks)' if args.hess_mode == 'dense' else ''} -> BSR over "
            f"2x388x388 two-sheet index space (stencils of each type in cell order) -> {PCG_ITERS} PCG iterations")


# ----------------------------------------------------------------------------- clocks
class ClockSampler:
    def __init__(self):
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-f", self.path],
                                         stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, device_index=0):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        try:
            with open(self.path) as f:
                for line in f:
                    parts = [p.strip() for p in line.split(",")]
                    if len(parts) >= 9 and parts[0] == str(device_index):
                        rows.append(parts)
            os.unlink(self.path)
        except Exception:
            return None
        if not rows:
            return None
        sm = sorted(float(r[1]) for r in rows)
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() in ("active", "1"):
                    reasons.add(nm)
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": float(rows[0][2]), "reasons": sorted(reasons),
                "samples": len(rows)}


# ----------------------------------------------------------------------------- GPU arm
def gpu_step(g, dev, W, args, bufs, ctx):
    import torch
    ev = torch.cuda.Event
    marks = [ev(enable_timing=True) for _ in range(4)]
    marks[0].record()
    eps = g.compute_eps_x(W["x"], W["st_own"], out=bufs["eps"])
    # dense blocks are written element-major as 3x3 sub-blocks (GIPC_HESS_BLOCKS): the same
    # values, contiguous for the assembly's per-contribution reads
    mode = "blocks" if args.hess_mode == "dense" else args.hess_mode
    e = g.eval_stencils(W["x"], W["st_own"], eps, W["dhat"], KAPPA, precision=args.precision,
                        mode=mode, want=("energy", "grad", "hess", "lam", "flags")
                        if args.hess_mode == "rank1" else ("energy", "grad", "hess", "flags"), out=bufs["eval"])
    bufs["eval"] = e
    marks[1].record()
    A = g.assemble_bsr(W["n"], stencils=W["st_sheet"], stencil_hess=e["hess"], stencil_mode=mode,
                       stencil_lam=e.get("lam"), stencil_grad=e["grad"], mass=W["mass"],
                       precision=args.precision, out=bufs["bsr"], ctx=ctx)
    bufs["bsr"] = {"rowptr": A["rowptr"], "colidx": A["colidx"], "vals": A["vals"], "grad": A["grad"]}
    marks[2].record()
    torch.neg(A["grad"], out=bufs["rhs"])
    d, k, rel = g.pcg(A, bufs["rhs"], rel_tol=0.0, max_iter=PCG_ITERS, ctx=ctx,
                      product=getattr(args, "product", "native"))
    marks[3].record()
    return d, A, marks


def e2e_pipelined(g, dev, W, Wh, args, bufs, ctx, steps, sync):
    """ms per step of the step through the public API with host inputs: every step copies its
    inputs (pinned host -> device) and reads its result back (device -> pinned host) inside the
    timed region.  The copies run on a second stream into two alternating input sets, so step k+1's
    inputs travel while step k computes (a pipeline a user with a stream of batches would run);
    the steps' computations themselves stay in order on the compute stream."""
    import torch
    keys = ("x", "st_own", "st_sheet", "mass")
    host = {k: torch.tensor(Wh[k]).pin_memory() for k in keys}
    out_h = torch.empty((3, Wh["n"]), dtype=torch.float64).pin_memory()
    sets = [{k: torch.empty_like(W[k]) for k in keys} for _ in range(2)]
    main, cs = torch.cuda.current_stream(), torch.cuda.Stream()
    copied = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def upload(b):
        with torch.cuda.stream(cs):
            for k in keys:
                sets[b][k].copy_(host[k], non_blocking=True)
            copied[b].record(cs)

    def pipeline(nsteps, start):
        cs.wait_event(start)
        upload(0)
        for k in range(nsteps):
            b = k % 2
            main.wait_event(copied[b])
            if k + 1 < nsteps:
                if k >= 1:
                    cs.wait_event(freed[1 - b])   # step k-1 has finished reading that set
                upload(1 - b)
            Wd = dict(W)
            Wd.update(sets[b])
            dd, _, _ = gpu_step(g, dev, Wd, args, bufs, ctx)
            freed[b].record(main)
            cs.wait_event(freed[b])
            dd.record_stream(cs)
            with torch.cuda.stream(cs):
                out_h.copy_(dd, non_blocking=True)
        main.wait_stream(cs)

    # untimed: the copy stream, the pinned buffers and the input sets go through the pipeline once
    sync()
    w0 = torch.cuda.Event()
    w0.record(main)
    pipeline(min(steps, 3), w0)
    sync()
    e0.record(main)
    pipeline(steps, e0)
    e1.record(main)
    sync()
    h2d = sum(t.numel() * t.element_size() for t in host.values())
    return e0.elapsed_time(e1) / steps, h2d, out_h.numel() * out_h.element_size()


def _scan_launches(m):
    """Kernels of one device-wide exclusive scan of m items (4096 per tile, recursive totals)."""
    return 1 if m <= 4096 else 2 + _scan_launches((m + 4095) // 4096)


def launches_per_step(n, nnzb, loop_launches_per_step):
    """The library's kernel launches in one C1 step (the sequence a launch list shows).

    eps_x + evaluation; assembly: row init, count, cursor init, fill, three row sorts, rowptr,
    emit, segment end, gradient init, the block-order histogram + scatter, values, two scans over
    the n rows and one over the 32 count bins x 1024-block chunks; solver: row-length
    histogram + scatter (+ scan of the 64 buckets x 1024-row chunks), slice lengths + fill (+ scan
    of the SELL-32 slices), scalars, two layout conversions, factors, the first product, setup, the
    final layout conversion, and the iterations: one persistent launch for all of them (the
    profiler's span count says whether it ran), else the product plus the fused update / direction
    per iteration."""
    order = (2 + _scan_launches(32 * ((nnzb + 1023) // 1024))) if nnzb > 0 else 0
    scans = 2 * _scan_launches(n) + _scan_launches(64 * ((n + 1023) // 1024)) + _scan_launches((n + 31) // 32)
    solver = 1 if loop_launches_per_step >= 1 else 2 * PCG_ITERS
    return 2 + 12 + order + 11 + scans + solver


def source_hash(*rel):
    h = hashlib.sha256()
    for r in rel:
        with open(os.path.join(ROOT, r), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, precision):
    """DRAM bytes per launch from a committed ncu summary, if it was taken on the current source."""
    try:
        with open(os.path.join(ROOT, "profiles", "traffic.json")) as f:
            T = json.load(f)
        ent = T[f"{kernel}/{precision}"]
        if ent["source_sha"] != source_hash(*ent["sources"]):
            return None
        return float(ent["dram_bytes_per_launch"])
    except Exception:
        return None


def run_gpu(args):
    import numpy as np
    import torch
    import torch.distributed as dist
    import paper_2308_09400_gb300 as g

    world, rank, local = rank_env()
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    ctx = g.default_context()
    for kind in ("pcg_spmv", "pcg_update", "pcg_direction"):   # spans on 1 of every PROF_EVERY iterations
        ctx.profile_sampling(kind, PROF_EVERY)

    Wh = workload(seed_offset=rank)
    W = {"x": torch.tensor(Wh["x"], device=dev), "st_own": torch.tensor(Wh["st_own"], device=dev),
         "st_sheet": torch.tensor(Wh["st_sheet"], device=dev), "mass": torch.tensor(Wh["mass"], device=dev),
         "n": Wh["n"], "dhat": Wh["dhat"]}
    bufs = {"eps": torch.empty(K_STENCILS, dtype=torch.float64, device=dev), "eval": {},
            "bsr": {}, "rhs": torch.empty((3, Wh["n"]), dtype=torch.float64, device=dev)}

    def barrier():
        if world > 1:
            dist.barrier()
        torch.cuda.synchronize()

    # warm-up (also sizes every buffer)
    for _ in range(args.warmup):
        d, A, _ = gpu_step(g, dev, W, args, bufs, ctx)
    barrier()

    clocks = ClockSampler()
    clocks.start()
    ctx.profile_begin()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    phase = np.zeros(3)
    barrier()
    t0.record()
    all_marks = []
    for _ in range(args.steps):
        d, A, marks = gpu_step(g, dev, W, args, bufs, ctx)
        all_marks.append(marks)
    t1.record()
    barrier()
    prof = ctx.profile_read()
    ctx.profile_stop()
    clk = clocks.stop(local)
    nnzb = A["nnzb"]
    ms = t0.elapsed_time(t1) / args.steps
    for m in all_marks:
        phase += [m[0].elapsed_time(m[1]), m[1].elapsed_time(m[2]), m[2].elapsed_time(m[3])]
    phase /= args.steps
    ms = max_over_ranks(ms, world, dev)

    # e2e: host (pinned) inputs in, Newton direction out, through the public API
    ctx.profile_begin()   # same per-kernel event spans as the timed region
    e2e_ms, h2d, d2h = e2e_pipelined(g, dev, W, Wh, args, bufs, ctx, args.steps, barrier)
    ctx.profile_stop()
    e2e_ms = max_over_ranks(e2e_ms, world, dev)

    if rank == 0:
        n = Wh["n"]
        roof = solver_roofline(prof, args.precision, n, nnzb)
        line = {
            "metric": METRIC, "value": job_rate(K_STENCILS, world, ms), "unit": "stencils/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
            "config": {"workload": workload_desc(args), "stencils_per_gpu": K_STENCILS, "vertices": n,
                       "nnzb": nnzb, "pcg_iterations": PCG_ITERS, "precision": args.precision,
                       "hess_mode": args.hess_mode, "parallelism": f"replicas{world}",
                       "l2": "inputs larger than L2 (>1.3 GB touched per step; no flush needed)",
                       "kernel_timing": f"CUDA-event spans in the timed region; PCG kernels on 1 of every {PROF_EVERY} "
                                        "iterations"},
            "phases_ms": {"eval": phase[0], "assemble": phase[1], "pcg": phase[2]},
            "kernel_ms": {k: (v[1] / max(v[0], 1)) for k, v in prof.items()},
            "linearize_solve_per_s": 1000.0 / ms,
            "roofline": roof,
            "e2e": {"value": job_rate(K_STENCILS, world, e2e_ms), "unit": "stencils/s", "h2d_bytes_per_step": h2d,
                    "d2h_bytes_per_step": d2h, "ms_per_step": e2e_ms},
            "gpu_launches": launches_per_step(n, nnzb, prof["pcg_loop"][0] / args.steps) * args.steps,
            "solver_phases_us": solver_phases(g, dev, W, args, bufs, ctx) if prof["pcg_loop"][0] else None,
            "clocks": clk,
        }
        if args.precision == "fp64" and args.hess_mode == "dense" and args.product == "native":
            line["float_pair_product"] = run_float_pair(g, dev, W, args, bufs, ctx)
            line["mixed"] = run_mixed(g, dev, W, Wh, args, ctx)
        if args.newton_steps > 0:
            line["newton"] = run_newton(g, dev, ctx, args.newton_steps, args.c2_steps)
        if args.batch_steps > 0:
            line["batched"] = run_batch_bench(g, dev, ctx, args.batch_steps)
        if args.diff_steps > 0:
            line["differentiation"] = run_diff_bench(g, dev, ctx, args.diff_steps)
            line["beam_plate"] = run_beam_forms(g, dev, args.diff_steps)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = cpu_baseline(args, Wh)
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()


# Algorithmic work of one solver iteration (FP64 flops count an FMA as two):
#   product: 9 FMA per block (18 flops), per row 3 adds + 3 FMA for a0 + a1 and c . q (9 flops);
#   vector phases per vertex: x += alpha c, r -= alpha q (12), the LDL^T solve and r . s (20),
#   the partial sum (1), c = s + beta c (6): 39 flops;
#   bytes: per block its values and column index, per row perm (4), q written (24) and c read
#   (24); per vertex c, q, x, r read (96), the factors (48 FP64 / 24 float32), x, r, c written
#   (72), and in the mixed form the float32 direction read and written (24).
def iteration_work(precision, n, nnzb):
    vb = 8 if precision == "fp64" else 4
    flops = 18 * nnzb + 9 * n + 39 * n
    bytes_ = nnzb * (9 * vb + 4) + n * (4 + 24 + 24) + n * (96 + (48 if precision == "fp64" else 24) + 72 +
                                                           (0 if precision == "fp64" else 24))
    return flops, bytes_


def solver_roofline(prof, precision, n, nnzb, kernel=None):
    """Roofline of the solver, the dominant kernel: algorithmic work of PCG_ITERS iterations over the
    mean CUDA-event duration of the persistent solver launch (one per step); FP64 against the FP64
    pipe, the mixed form against measured HBM bandwidth."""
    hbm, hbm_src = peaks()
    loop_n, loop_ms = prof["pcg_loop"]
    flops_it, bytes_it = iteration_work(precision, n, nnzb)
    if loop_n > 0:
        avg = loop_ms / loop_n * 1e-3
        its = PCG_ITERS
        name = kernel or ("pcg_loop_kernel<double, double, 1, 2, false>" if precision == "fp64"
                          else "pcg_loop_kernel<float, float, 2, 2, true>")
    else:   # (fallback path) product + fused update per iteration, from their sampled spans
        sp, up = prof["pcg_spmv"], prof["pcg_update"]
        avg = (sp[1] / max(sp[0], 1) + up[1] / max(up[0], 1)) * 1e-3
        its = 1
        name = "pcg_spmv_tma_kernel + pcg_update_direction_kernel"
    ach_fl = flops_it * its / avg / 1e9
    ach_bw = bytes_it * its / avg / 1e9
    if precision == "fp64":
        roof = {"bound": "alu", "achieved": ach_fl / 1e3, "peak": FP64_PEAK / 1e3, "unit": "TFLOP/s",
                "frac": ach_fl / FP64_PEAK,
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2070 MHz (an FMA probe measured 1.19-1.26 TFLOP/s)",
                "hbm_frac": ach_bw / hbm}
    else:
        roof = {"bound": "hbm", "achieved": ach_bw, "peak": hbm, "unit": "GB/s", "frac": ach_bw / hbm,
                "peak_source": f"{hbm_src} (MEASURED_PEAKS.json hbm_gbs)" if hbm_src == "measured" else hbm_src}
    roof.update({"kernel": name, "launch_us": avg * 1e6, "iterations_per_launch": its,
                 "us_per_iteration": avg * 1e6 / its, "algorithmic_flops_per_iteration": flops_it,
                 "algorithmic_bytes_per_iteration": bytes_it, "launches": loop_n,
                 "traffic": measured_traffic("pcg_loop", precision)})
    return roof


def solver_phases(g, dev, W, args, bufs, ctx):
    """One more C1 step with the persistent solver's phase stamps on (outside the timed region):
    the median length of each phase of an iteration, in microseconds."""
    ctx.solver_trace(True)
    try:
        gpu_step(g, dev, W, args, bufs, ctx)
        ph, its = ctx.solver_phases()
    finally:
        ctx.solver_trace(False)
    ph["iterations_used"] = its
    return ph


def timed_steps(g, dev, W, args, bufs, ctx, steps):
    """`steps` C1 steps after two untimed ones: ms per step and the profiler's spans."""
    import torch
    for _ in range(2):
        gpu_step(g, dev, W, args, bufs, ctx)
    torch.cuda.synchronize()
    ctx.profile_begin()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(steps):
        d, A, marks = gpu_step(g, dev, W, args, bufs, ctx)
    e1.record()
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile_stop()
    return e0.elapsed_time(e1) / steps, prof, d, A, marks


def run_float_pair(g, dev, W, args, bufs, ctx):
    """The same C1 step with the solver's H c in double-float arithmetic (gipc_product
    GIPC_PRODUCT_FLOAT_PAIR): time per step, the solver against the HBM roof (same bytes as FP64),
    and the Newton direction's deviation from the native FP64 result after the same iterations."""
    import argparse
    a2 = argparse.Namespace(**dict(vars(args), product="float_pair"))
    d_native, _, _ = gpu_step(g, dev, W, args, bufs, ctx)   # the native solve of the same inputs
    d_native = d_native.clone()
    ms, prof, d2, A, _ = timed_steps(g, dev, W, a2, bufs, ctx, args.steps)
    import torch
    ok = bool(torch.isfinite(d_native).all().item()) and bool(torch.isfinite(d2).all().item())
    dev_rel = ((d2 - d_native).abs().max() / d_native.abs().max()).item() if ok else float("nan")
    roof = solver_roofline(prof, "fp64", W["n"], A["nnzb"], kernel="pcg_loop_kernel<fpair, fpair, 2, 2, false>")
    return {"ms_per_step": ms, "stencils_per_s": K_STENCILS / (ms * 1e-3),
            "solver_us_per_iteration": roof["us_per_iteration"], "solver_hbm_frac": roof["hbm_frac"],
            "kernel": roof["kernel"],
            "direction_max_rel_dev_from_native": dev_rel,
            "note": "FP64 matrix and vectors; H c products and sums as float32 pairs (about 2^-44 relative "
                    "per row); not the headline"}


def run_mixed(g, dev, W, Wh, args, ctx):
    """The mixed form of the same C1 step (float32 rank-one blocks, BSR, product, factors and
    direction; FP64 distances, barrier log, mollifier, residual and dots): time per step, stencils
    per second, end to end with host inputs, the solver's HBM roofline, the per-block relative
    Frobenius error of the mixed Hessian blocks against the FP64 path's (which matches the oracle to
    1e-10 in the tests) over all 1M stencils."""
    import argparse
    import torch
    a2 = argparse.Namespace(**dict(vars(args), precision="mixed", hess_mode="rank1"))
    bufs = {"eps": torch.empty(K_STENCILS, dtype=torch.float64, device=dev), "eval": {}, "bsr": {},
            "rhs": torch.empty((3, Wh["n"]), dtype=torch.float64, device=dev)}
    ms, prof, d, A, marks = timed_steps(g, dev, W, a2, bufs, ctx, args.steps)
    roof = solver_roofline(prof, "mixed", Wh["n"], A["nnzb"])
    phases = solver_phases(g, dev, W, a2, bufs, ctx) if prof["pcg_loop"][0] else None
    # end to end: host inputs in, direction out
    e2e_ms, _, _ = e2e_pipelined(g, dev, W, Wh, a2, bufs, ctx, args.steps, torch.cuda.synchronize)
    # per-block error: mixed rank-one blocks lam w w^T (float32) against the FP64 dense blocks
    eps = g.compute_eps_x(W["x"], W["st_own"])
    f64 = g.eval_stencils(W["x"], W["st_own"], eps, W["dhat"], KAPPA, precision="fp64", mode="rank1",
                          want=("hess", "lam"))
    mx = g.eval_stencils(W["x"], W["st_own"], eps, W["dhat"], KAPPA, precision="mixed", mode="rank1",
                         want=("hess", "lam"))
    w64, l64 = f64["hess"].double(), f64["lam"].double()
    w32, l32 = mx["hess"].double(), mx["lam"].double()
    # ||l32 w32 w32^T - l64 w64 w64^T||_F / ||l64 w64 w64^T||_F, via inner products (no dense blocks)
    a2n = (w32 * w32).sum(0)
    b2n = (w64 * w64).sum(0)
    ab = (w32 * w64).sum(0)
    num2 = (l32 * a2n) ** 2 + (l64 * b2n) ** 2 - 2 * l32 * l64 * ab ** 2
    den = (l64 * b2n).abs()
    act = den > 0
    rel = torch.sqrt(num2[act].clamp_min(0)) / den[act]
    return {"ms_per_step": ms, "value": K_STENCILS / (ms * 1e-3), "unit": "stencils/s",
            "e2e": {"value": K_STENCILS / (e2e_ms * 1e-3), "unit": "stencils/s", "ms_per_step": e2e_ms},
            "phases_ms": {"eval": marks[0].elapsed_time(marks[1]), "assemble": marks[1].elapsed_time(marks[2]),
                          "pcg": marks[2].elapsed_time(marks[3])},
            "roofline": roof, "solver_phases_us": phases, "dtype": "f32+f64", "hess_mode": "rank1",
            "block_rel_frobenius_err_vs_fp64": {"max": rel.max().item(), "mean": rel.mean().item(),
                                                "blocks": int(act.sum().item()), "bar": 1e-4},
            "note": "same inputs and iteration count as the FP64 line (200 iterations at tolerance 0 on a "
                    "system with diagonal blocks of condition ~1e12, so the two forms' iterates are not "
                    "compared); the converged-position error of the mixed form is under "
                    "newton.converged_position_error"}


# ----------------------------------------------------------------------------- Newton iterations/s
NEWTON_FORMS = (("fp64", "dense"), ("mixed", "rank1"))


def newton_scene():
    """8 x 8 tet-meshed spheres (radius 0.1, 14 cells per diameter) 1e-3 above a tessellated
    floor slab and 1e-3 apart; E = 1e5 Pa, nu = 0.4, rho = 1000, dt = 0.01, dhat = 1e-3 l,
    kappa = 1e3, gravity -9.81 z."""
    import synth
    return synth.sphere_grid(8, 8)


def run_c2(g, scene, sc, prm, dev, steps):
    """Converged-position error of the mixed rank-one form against FP64 dense.  After one FP64
    settling step (the initially compressed lattice has several nearby minima, so that first step
    lands on a path-dependent one in any precision), each step starts from the FP64 state and is
    solved by both forms to eps_d = 1e-5 (PCG tolerance 1e-7); the FP64 result carries the
    trajectory on.  Reported per step as max |x_mixed - x_fp64| / l."""
    import numpy as np
    import torch
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    tight = dict(prm, eps_d=1e-5, pcg_tol=1e-7, max_pcg=5000, max_newton=200)
    x, v = T(sc["x"]), T(sc["v"])
    g.newton_step(scene, x, v, precision="fp64", hess_mode="dense", **tight)
    errs, conv, iters = [], [], []
    for _ in range(steps):
        out = {}
        for prec, hm in NEWTON_FORMS:
            xx, vv = x.clone(), v.clone()
            st = g.newton_step(scene, xx, vv, precision=prec, hess_mode=hm, **tight)
            out[prec] = (xx, vv, st)
        errs.append((out["mixed"][0] - out["fp64"][0]).abs().max().item() / sc["l"])
        conv.append([out["fp64"][2]["converged"], out["mixed"][2]["converged"]])
        iters.append([out["fp64"][2]["newton_iters"], out["mixed"][2]["newton_iters"]])
        x, v = out["fp64"][0], out["fp64"][1]
    return {"definition": "after one FP64 settling step; per step, from the FP64 state: "
                          "max|x_mixed - x_fp64| / l, both solved to eps_d 1e-5, PCG tol 1e-7",
            "max_err_over_l": max(errs), "per_step_err_over_l": errs, "converged_fp64_mixed": conv,
            "newton_iters_fp64_mixed": iters, "target": 1e-6}


def run_newton(g, dev, ctx, steps, c2_steps=0):
    """Implicit time steps of the sphere-grid scene through gipc_newton_step, FP64 dense and mixed
    rank-one forms from the same initial state; Newton iterations per second and per-phase times."""
    import numpy as np
    import torch

    sc = newton_scene()
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    srf = g.Surface(T(sc["tris"]), T(sc["edges"]), T(sc["verts"]))
    scene = g.Scene(T(sc["x"]), T(sc["tets"]), srf, 1000.0, fixed=T(sc["fixed"]), l=sc["l"])
    mu, lam = g.snh_params(1e5, 0.4)
    prm = dict(dt=0.01, mu=mu, lam=lam, dhat=1e-3 * sc["l"], kappa=KAPPA, eps_d=1e-2, pcg_tol=1e-4,
               max_pcg=1000, max_newton=50)
    out = {"scene": {"workload": "sphere grid 8x8 (radius 0.1) on a tessellated floor slab",
                     "vertices": int(sc["x"].shape[1]), "tets": int(sc["tets"].shape[1]),
                     "surface_tris": int(sc["tris"].shape[1]), "surface_edges": int(sc["edges"].shape[1]),
                     "dt": 0.01, "dhat": prm["dhat"], "kappa": KAPPA, "eps_d": 1e-2, "pcg_tol": 1e-4,
                     "E": 1e5, "nu": 0.4, "rho": 1000.0}}
    for prec, hm in NEWTON_FORMS:
        x, v = T(sc["x"]), T(sc["v"])
        g.newton_step(scene, x, v, precision=prec, hess_mode=hm, **prm)   # warm-up step (sizes scratch)
        torch.cuda.synchronize()
        ctx.profile_begin()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = pcg = 0
        e0.record()
        for _ in range(steps):
            st = g.newton_step(scene, x, v, precision=prec, hess_mode=hm, **prm)
            iters += st["newton_iters"]
            pcg += st["pcg_iters"]
        e1.record()
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile_stop()
        ms = e0.elapsed_time(e1)
        # the solver kernels' spans are sampled: mean span x launches (one per PCG iteration)
        phase = {k: (v[1] / max(v[0], 1) * pcg if k in ("pcg_spmv", "pcg_update") else v[1]) / max(iters, 1)
                 for k, v in prof.items() if k != "pcg_direction"}
        out[f"{prec}_{hm}"] = {"newton_iters_per_s": iters / (ms * 1e-3), "ms_per_newton_iter": ms / max(iters, 1),
                               "time_steps": steps, "newton_iters": iters, "pcg_iters": pcg,
                               "contacts_final": st["contacts"], "phase_ms_per_newton_iter": phase}
    if c2_steps > 0:
        out["converged_position_error"] = run_c2(g, scene, sc, prm, dev, c2_steps)
    return out


def run_beam_forms(g, dev, steps):
    """Implicit time steps of the beam-on-plate scene (the differentiation workload) through
    gipc_newton_step in the FP64 dense and mixed rank-one forms, from the same initial state, at
    the forward settings of the sphere-grid scene (eps_d 1e-2, PCG tol 1e-4, no refinement)."""
    import numpy as np
    import torch
    import synth

    sc = synth.beam_on_plate(dhat_rel=BEAM_DHAT_REL)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    srf = g.Surface(T(sc["tris"]), T(sc["edges"]), T(sc["verts"]))
    scene = g.Scene(T(sc["x"]), T(sc["tets"]), srf, 1000.0, fixed=T(sc["fixed"]), l=sc["l"])
    mu, lam = g.snh_params(1e5, 0.4)
    prm = dict(dt=0.01, mu=mu, lam=lam, dhat=sc["dhat"], kappa=KAPPA, eps_d=1e-2, pcg_tol=1e-4,
               max_pcg=1000, max_newton=50)
    out = {"workload": f"tet beam 41x11x11 on a tet plate 65x65x4 (the differentiation scene), dhat = {BEAM_DHAT_REL} l",
           "vertices": int(sc["x"].shape[1]), "tets": int(sc["tets"].shape[1]), "eps_d": 1e-2, "pcg_tol": 1e-4}
    for prec, hm in NEWTON_FORMS:
        x, v = T(sc["x"]), T(sc["v"])
        g.newton_step(scene, x.clone(), v.clone(), precision=prec, hess_mode=hm, **prm)   # warm-up
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        iters = pcg = 0
        e0.record()
        for _ in range(steps):
            st = g.newton_step(scene, x, v, precision=prec, hess_mode=hm, **prm)
            iters += st["newton_iters"]
            pcg += st["pcg_iters"]
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1)
        out[f"{prec}_{hm}"] = {"newton_iters_per_s": iters / (ms * 1e-3), "ms_per_newton_iter": ms / max(iters, 1),
                               "time_steps": steps, "newton_iters": iters, "pcg_iters": pcg,
                               "contacts_final": st["contacts"]}
    return out


# ----------------------------------------------------------------------------- batched scenes
def run_batch_bench(g, dev, ctx, steps):
    """256 independent scenes (2-6 stacked cubes / balls each, 200-5000 vertices log-uniform, gaps
    uniform in [0, 2 dhat]): `steps` implicit steps from rest through gipc_newton_step_batch, and the
    same steps of every scene alone through gipc_newton_step; scene Newton iterations per second."""
    import numpy as np
    import torch
    import synth

    scenes, dhat = synth.batch_scenes(256)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    mu, lam = g.snh_params(1e5, 0.4)
    prm = dict(dt=0.01, mu=mu, lam=lam, dhat=dhat, kappa=KAPPA, eps_d=1e-2, pcg_tol=1e-4, max_pcg=1000,
               max_newton=50)
    b = g.SceneBatch(scenes, 1000.0)
    v_init = np.concatenate([sc["v"] for sc in scenes], axis=1)
    singles = []
    for sc in scenes:
        srf = g.Surface(T(sc["tris"]), T(sc["edges"]), T(sc["verts"]))
        singles.append(g.Scene(T(sc["x"]), T(sc["tets"]), srf, 1000.0, fixed=T(sc["fixed"]), l=sc["l"]))
    out = {"workload": "256 scenes of 2-6 stacked tet cubes / balls, 200-5000 vertices each (log-uniform), "
                       "gaps uniform in [0, 2 dhat]",
           "vertices": int(sum(sc["x"].shape[1] for sc in scenes)), "tets": int(sum(sc["tets"].shape[1] for sc in scenes)),
           "dhat": dhat, "time_steps": steps}
    for prec, hm in NEWTON_FORMS:
        # warm-up (scratch sizing) on a throw-away copy
        xw, vw = b.scene.rest_x.clone(), T(v_init)
        g.newton_step_batch(b, xw, vw, precision=prec, hess_mode=hm, **prm)
        x, v = b.scene.rest_x.clone(), T(v_init)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        marks = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
        e0.record()
        its = 0
        per_step, longest = [], []
        for i in range(steps):
            st = g.newton_step_batch(b, x, v, precision=prec, hess_mode=hm, **prm)
            marks[i].record()
            per_step.append(sum(s["newton_iters"] for s in st))
            longest.append(max(s["newton_iters"] for s in st))
        e1.record()
        torch.cuda.synchronize()
        ms_b = e0.elapsed_time(e1)
        step_ms = [e0.elapsed_time(marks[0])] + [marks[i - 1].elapsed_time(marks[i]) for i in range(1, steps)]
        its = sum(per_step)
        # the same batched steps once more with the phase spans on (outside the timed region)
        xp, vp = b.scene.rest_x.clone(), T(v_init)
        torch.cuda.synchronize()
        ctx.profile_begin()
        for _ in range(steps):
            g.newton_step_batch(b, xp, vp, precision=prec, hess_mode=hm, **prm)
        torch.cuda.synchronize()
        prof = ctx.profile_read()
        ctx.profile_stop()
        phases = {k: v[1] / steps for k, v in prof.items() if v[0] and k not in ("pcg_spmv", "pcg_update", "pcg_direction")}
        pcg_spans = {k: {"spans": v[0], "mean_us": v[1] / v[0] * 1e3} for k, v in prof.items()
                     if v[0] and k in ("pcg_spmv", "pcg_update", "pcg_direction")}
        # the same steps, every scene alone
        xs = [T(sc["x"]) for sc in scenes]
        vs = [T(sc["v"]) for sc in scenes]
        g.newton_step(singles[0], xs[0].clone(), vs[0].clone(), precision=prec, hess_mode=hm, **prm)
        torch.cuda.synchronize()
        e0.record()
        its1 = 0
        for _ in range(steps):
            for k in range(len(scenes)):
                its1 += g.newton_step(singles[k], xs[k], vs[k], precision=prec, hess_mode=hm, **prm)["newton_iters"]
        e1.record()
        torch.cuda.synchronize()
        ms_p = e0.elapsed_time(e1)
        # the product's staging variant the run-time tuner chose per size class of the batch (the
        # classes shrink as finished scenes are packed out)
        tuning = []
        for t in ctx.spmv_tunings():
            if t["precision"] != prec:
                continue
            name = lambda v: f"U{v['U']}_W{v['W']}_NS{v['NS']}"
            tuning.append({"size_class_log2_nnzb": t["size_class"],
                           "chosen": name(t["variants"][t["chosen"]]) if t["chosen"] >= 0 else None,
                           "mean_us": {name(v): round(v["mean_us"], 2) for v in t["variants"]},
                           "samples": [v["samples"] for v in t["variants"]]})
        out[f"{prec}_{hm}"] = {"batched_ms_per_step": ms_b / steps, "batched_scene_iters_per_s": its / (ms_b * 1e-3),
                               "one_at_a_time_ms_per_step": ms_p / steps,
                               "one_at_a_time_scene_iters_per_s": its1 / (ms_p * 1e-3),
                               "scene_newton_iters": its, "scene_newton_iters_one_at_a_time": its1,
                               "scene_newton_iters_per_step": per_step, "batched_iters_per_step": longest,
                               "batched_ms_each_step": step_ms,
                               "speedup": ms_p / ms_b,
                               "phase_ms_per_step": phases, "pcg_kernel_spans": pcg_spans,
                               "solver": ("one persistent launch per solve" if "pcg_loop" in phases
                                          else "a product and a per-scene update launch per iteration"),
                               "product_variant_tuning": tuning}
    return out


# ----------------------------------------------------------------------------- differentiation
DIFF_SEED = 20230814
# dhat of the beam-on-plate scene relative to its bounding-box diagonal.  The scene is described by
# its contact load (about 30k contact stencils); its meshes reach that at the start near 6.5e-3 l
# (initial contacts: 1e-3 l: 5.1k, 5e-3 l: 14.7k, 7e-3 l: 36.6k), but there the exact Hessian of
# the projected-Newton result is indefinite and its refinement stalls at 3.7e-6 l dt, so the
# differentiated steps use 5e-3 l: 14.7k contacts at the start, about 6k through the steps.
BEAM_DHAT_REL = 5e-3


def run_diff_bench(g, dev, ctx, steps, fd_h=1e-6, eps_d=1e-5, eps_polish=1e-12, polish_iters=30, dhat_rel=None):
    """Tet beam (41 x 11 x 11 vertices, 1.0 x 0.25 x 0.25) turned 0.3 rad about z and resting on a
    tet plate (65 x 65 x 4 vertices, 2 x 2, bottom layer fixed), the beam moving at (0.05, 0, -0.1)
    m/s; FP64 dense steps (dt 0.01, E 1e5, nu 0.4, rho 1000, dhat 1e-3 l, kappa 1e3).
    Each step: projected Newton to eps_d, then exact-Hessian Newton refinement to eps_polish.
    L = w . x_T for seeded w: `steps` checkpointed steps, the implicit adjoint back through them
    (dL/dv0, E dL/dE), the exact derivative kernels at x_T (gradient + Hessian-vector product per
    element and through autograd), and central differences with step fd_h of L along a seeded
    direction of v0 and in log E."""
    import numpy as np
    import torch
    import synth

    sc = synth.beam_on_plate(dhat_rel=dhat_rel or BEAM_DHAT_REL)
    T = lambda a: torch.tensor(np.ascontiguousarray(a), device=dev)
    srf = g.Surface(T(sc["tris"]), T(sc["edges"]), T(sc["verts"]))
    scene = g.Scene(T(sc["x"]), T(sc["tets"]), srf, 1000.0, fixed=T(sc["fixed"]), l=sc["l"])
    mu, lam = g.snh_params(1e5, 0.4)
    dt, dhat = 0.01, sc["dhat"]
    prm = dict(dt=dt, mu=mu, lam=lam, dhat=dhat, kappa=KAPPA, eps_d=eps_d, pcg_tol=1e-10, max_pcg=5000,
               max_newton=100)
    pol = dict(eps_polish=eps_polish, max_iters=polish_iters, pcg_tol=1e-24, max_pcg=20000)
    adj_tol = 1e-22     # r.P^-1 r relative to its start: an 1e-11 smaller residual
    x0, v0 = T(sc["x"]), T(sc["v"])
    g.newton_step(scene, x0.clone(), v0.clone(), **prm)      # warm-up (scratch sizing)
    torch.cuda.synchronize()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    e0, e1 = ev(), ev()
    stats = []
    e0.record()
    xT, vT, cps = g.simulate(scene, x0, v0, steps, stats=stats, polish=pol, **prm)
    e1.record()
    torch.cuda.synchronize()
    fwd_ms = e0.elapsed_time(e1)
    rng = np.random.default_rng(DIFF_SEED)
    w = T(rng.normal(size=sc["x"].shape))
    zero = torch.zeros_like(w)
    g.adjoint_step(scene, cps[1][0], cps[0][0], cps[0][1], w, zero, dt, mu, lam, dhat, KAPPA, pcg_tol=adj_tol,
                   max_pcg=20000)
    torch.cuda.synchronize()
    e0.record()
    ax0, av0, logE, its = g.adjoint(scene, cps, w, zero, dt, mu, lam, dhat, KAPPA, pcg_tol=adj_tol, max_pcg=20000)
    e1.record()
    torch.cuda.synchronize()
    adj_ms = e0.elapsed_time(e1)

    # derivative kernels at x_T with the contacts there
    stn, eps = g.find_contacts(xT, scene.rest_x, scene.surface, dhat)
    k = int(stn.shape[1])
    ntet = int(sc["tets"].shape[1])
    xt = cps[-2][0] + dt * cps[-2][1]
    u = T(rng.normal(size=sc["x"].shape))
    args = (scene, xT, stn, eps, dhat, KAPPA, mu, lam, dt * dt)
    reps = 20
    for _ in range(3):
        g.potential_derivs(*args, xt=xt, u=u, want=("grad",))
    torch.cuda.synchronize()
    e0.record()
    for _ in range(reps):
        g.potential_derivs(*args, xt=xt, u=u, want=("grad",))
    e1.record()
    torch.cuda.synchronize()
    derivs_ms = e0.elapsed_time(e1) / reps
    X = xT.clone().requires_grad_(True)
    for r in range(reps + 3):
        if r == 3:
            torch.cuda.synchronize()
            e0.record()
        I = g.incremental_potential(X, scene, xt, stn, eps, dhat, KAPPA, mu, lam, dt * dt)
        (gX,) = torch.autograd.grad(I, X, create_graph=True)
        (Hu,) = torch.autograd.grad((gX * u).sum(), X)
    e1.record()
    torch.cuda.synchronize()
    autograd_ms = e0.elapsed_time(e1) / reps

    # central differences of the GPU forward
    def L(v, mu_=mu, lam_=lam):
        xx, _, _ = g.simulate(scene, x0, v, steps, polish=pol, **dict(prm, mu=mu_, lam=lam_))
        return float((w * xx).sum())

    dirv = rng.normal(size=sc["x"].shape)
    dirv[:, np.asarray(sc["fixed"], bool)] = 0.0
    dv = T(dirv)
    fd_v = (L(v0 + fd_h * dv) - L(v0 - fd_h * dv)) / (2 * fd_h)
    ad_v = float((av0 * dv).sum())
    mp, lp = g.snh_params(1e5 * (1 + fd_h), 0.4)
    mm, lm = g.snh_params(1e5 * (1 - fd_h), 0.4)
    fd_E = (L(v0, mp, lp) - L(v0, mm, lm)) / (np.log1p(fd_h) - np.log1p(-fd_h))
    newton_its = sum(s["newton_iters"] for s in stats)
    return {"workload": f"tet beam 41x11x11 (turned 0.3 rad) resting on a tet plate 65x65x4, dhat = {BEAM_DHAT_REL} l, beam at "
                        "(0.05, 0, -0.1) m/s; L = w . x_T, w seeded normal",
            "vertices": int(sc["x"].shape[1]), "tets": ntet, "surface_tris": int(sc["tris"].shape[1]),
            "surface_edges": int(sc["edges"].shape[1]), "dhat": dhat, "eps_d": eps_d, "eps_polish": eps_polish,
            "time_steps": steps, "polish_iters": [s["polish_iters"] for s in stats],
            "polish_final_step": max(s["polish_step"] for s in stats),
            "contacts_per_step": [s["contacts"] for s in stats], "newton_iters": newton_its,
            "converged_steps": int(sum(s["converged"] for s in stats)),
            "forward_ms": fwd_ms,
            "forward_iters_per_s": (newton_its + sum(s["polish_iters"] for s in stats)) / (fwd_ms * 1e-3),
            "adjoint_ms": adj_ms, "adjoint_ms_per_step": adj_ms / steps, "adjoint_pcg_iters": its,
            "adjoint_pcg_tol": adj_tol,
            "derivative_kernels": {"contacts": k, "tets": ntet, "grad_and_hvp_ms": derivs_ms,
                                   "elements_per_s": (k + ntet) / (derivs_ms * 1e-3),
                                   "autograd_grad_and_double_backward_ms": autograd_ms},
            "fd_check": {"h": fd_h, "dL_dv0_dir": {"adjoint": ad_v, "fd": fd_v,
                                                   "rel_err": abs(ad_v - fd_v) / abs(fd_v)},
                         "E_dL_dE": {"adjoint": logE, "fd": fd_E, "rel_err": abs(logE - fd_E) / abs(fd_E)}}}


# ----------------------------------------------------------------------------- oracle (CPU) arm
ORACLE_EVAL_SAMPLE = 400       # stencils evaluated per measurement (one core, in process)
ORACLE_ASM_SAMPLE = 2000       # stencils assembled per measurement (their own compact index space)
ORACLE_MASS_ROWS = 20000       # mass rows assembled per measurement
ORACLE_PCG_ITERS = 10         # oracle PCG iterations timed per measurement (tolerance 0: equal cost each)


def full_pattern_system(Wh):
    """A BSR system of the benchmark's full size and pattern (4.1M blocks over 301,088 rows) for
    timing the oracle's solver: mass on the diagonal plus a rank-one PSD block per stencil, summed
    per block by numpy from the stencils' plain vertex tuples (not by the library; the solver's cost
    does not depend on the values)."""
    import numpy as np
    n = Wh["n"]
    rng = np.random.default_rng(20230815)
    rows, cols = [np.arange(n, dtype=np.int64)], [np.arange(n, dtype=np.int64)]
    contrib = [np.asarray(Wh["mass"])[:, None, None] * np.eye(3)]
    for ids in Wh["sheet_ids"]:
        m, s = ids.shape
        w = rng.normal(size=(m, s, 3))
        lam = 10.0 ** rng.uniform(0, 4, m)
        for a in range(s):
            for b in range(s):
                rows.append(ids[:, a])
                cols.append(ids[:, b])
                contrib.append(lam[:, None, None] * w[:, a, :, None] * w[:, b, None, :])
    rows, cols = np.concatenate(rows), np.concatenate(cols)
    contrib = np.concatenate(contrib).reshape(-1, 9)
    key, inv = np.unique(rows * n + cols, return_inverse=True)
    vals = np.stack([np.bincount(inv, weights=contrib[:, e], minlength=len(key)) for e in range(9)], 1)
    rowptr = np.zeros(n + 1, np.int64)
    np.add.at(rowptr, key // n + 1, 1)
    return {"rowptr": np.cumsum(rowptr), "colidx": key % n, "vals": vals.reshape(-1, 3, 3)}, rng.normal(size=(3, n))


def full_stencil_keys(Wh):
    """Assembly keys of the whole batch's stencils: every ordered vertex pair of every stencil."""
    return sum(ids.shape[0] * ids.shape[1] ** 2 for ids in Wh["sheet_ids"])


def _decoded_ids(st):
    """Vertex ids of sign-encoded stencil tuples (negative slot -(i + 1), null slots dropped)."""
    import numpy as np
    v = np.asarray(st, dtype=np.int64)
    ids = np.where(v >= 0, v, -v - 1)
    return ids[v != -2147483648]


def _compact(st):
    """The tuples renumbered onto the vertices they use (signs and null slots kept)."""
    import numpy as np
    v = np.asarray(st, dtype=np.int64)
    null = v == -2147483648
    ids = np.where(v >= 0, v, -v - 1)
    uniq, inv = np.unique(np.where(null, -1, ids), return_inverse=True)
    shift = 1 if uniq[0] == -1 else 0
    new = inv.reshape(v.shape) - shift
    out = np.where(null, v, np.where(v >= 0, new, -new - 1))
    return np.ascontiguousarray(out.astype(np.int32)), len(uniq) - shift


def oracle_step_costs(args, Wh, system):
    """The oracle's cost of one C1 step from its costs per unit of work, each measured on one core
    in this process on a fixed amount of that work, so the result does not depend on sample sizes:
    the stencil evaluation per stencil (ORACLE_EVAL_SAMPLE stencils), the plain assembly per key
    (ORACLE_ASM_SAMPLE stencils over the vertices they use) and per mass row (ORACLE_MASS_ROWS
    rows), and the PCG per iteration (ORACLE_PCG_ITERS iterations at tolerance 0 on a full-size
    system of the benchmark's pattern).  Step = K x s per stencil + the batch's keys x s per key +
    n x s per row + PCG_ITERS x s per iteration."""
    import numpy as np
    from oracle import assembly as OA
    from oracle import pcg as OP
    from oracle import stencil as OS
    ke = ORACLE_EVAL_SAMPLE
    st = np.ascontiguousarray(Wh["st_own"][:, :ke])
    xs = np.ascontiguousarray(Wh["x"][:, :int(_decoded_ids(st).max()) + 1])
    eps = OS.compute_eps_x(xs, st)
    t = time.perf_counter()
    OS.eval_stencils(xs, st, eps, Wh["dhat"], KAPPA, processes=1)
    s_eval = (time.perf_counter() - t) / ke
    ka = ORACLE_ASM_SAMPLE
    sh, m = _compact(Wh["st_sheet"][:, :ka])
    rng = np.random.default_rng(20230816)
    if args.hess_mode == "rank1":
        sd = {"kind": "rank1", "lam": rng.uniform(1, 2, ka), "w": rng.normal(size=(12, ka)), "grad": rng.normal(size=(12, ka))}
    else:
        sd = {"kind": "dense", "hess": rng.normal(size=(144, ka)), "grad": rng.normal(size=(12, ka))}
    keys = sum(len(v) ** 2 for v in OA.element_vertices(sh, None))
    t = time.perf_counter()
    OA.assemble(m, sh, sd, None, None, None)
    s_key = (time.perf_counter() - t) / keys
    nr = ORACLE_MASS_ROWS
    t = time.perf_counter()
    OA.assemble(nr, None, None, None, None, np.asarray(Wh["mass"])[:nr])
    s_row = (time.perf_counter() - t) / nr
    R, b = system
    t = time.perf_counter()
    OP.pcg(R, Wh["n"], b, tol=0.0, max_iter=ORACLE_PCG_ITERS)
    s_it = (time.perf_counter() - t) / ORACLE_PCG_ITERS
    total = K_STENCILS * s_eval + full_stencil_keys(Wh) * s_key + Wh["n"] * s_row + PCG_ITERS * s_it
    return {"eval_stencils_per_s": 1.0 / s_eval, "assembly_keys_per_s": 1.0 / s_key, "mass_rows_per_s": 1.0 / s_row,
            "pcg_s_per_iteration": s_it, "full_step_s": total, "stencils_per_s": K_STENCILS / total}


def _oracle_desc(n, nnzb_full):
    return (f"oracle on one host core, its cost per unit of work scaled to the whole {K_STENCILS}-stencil step: "
            f"exact-geometry evaluation of {ORACLE_EVAL_SAMPLE} stencils (s per stencil x {K_STENCILS}), plain "
            f"assembly of {ORACLE_ASM_SAMPLE} stencils (s per key x the batch's keys) and of {ORACLE_MASS_ROWS} mass "
            f"rows (s per row x {n}), and {ORACLE_PCG_ITERS} oracle PCG iterations on a full-size system of the "
            f"benchmark's pattern ({nnzb_full} blocks; s per iteration x {PCG_ITERS})")


def cpu_baseline(args, Wh):
    """The oracle's whole step from its per-unit costs on one host core (see oracle_step_costs),
    and, for reference, its stencil evaluation alone on all host cores (spawned processes)."""
    import numpy as np
    from oracle import stencil as OS
    system = full_pattern_system(Wh)
    c = oracle_step_costs(args, Wh, system)
    procs = os.cpu_count() or 1
    k = 4000
    st = np.ascontiguousarray(Wh["st_own"][:, :k])
    xs = np.ascontiguousarray(Wh["x"][:, :int(_decoded_ids(st).max()) + 1])
    eps = OS.compute_eps_x(xs, st)
    t = time.perf_counter()
    OS.eval_stencils(xs, st, eps, Wh["dhat"], KAPPA, processes=procs)
    eval_all = k / (time.perf_counter() - t)
    return {"value": c["stencils_per_s"], "unit": "stencils/s", "cores": 1, "kind": "oracle",
            "sample": _oracle_desc(Wh["n"], len(system[0]["colidx"])),
            "phases": {"eval_stencils_per_s": c["eval_stencils_per_s"], "assembly_keys_per_s": c["assembly_keys_per_s"],
                       "mass_rows_per_s": c["mass_rows_per_s"], "pcg_s_per_iteration": c["pcg_s_per_iteration"],
                       "full_step_s": c["full_step_s"]},
            "eval_only_all_cores": {"stencils_per_s": eval_all, "cores": procs, "sample": k,
                                    "note": "pool start-up included"}}


def run_reference(args):
    world, rank, _ = rank_env()
    if rank != 0:
        return
    Wh = workload()
    system = full_pattern_system(Wh)
    for _ in range(args.warmup):
        oracle_step_costs(args, Wh, system)
    totals = []
    t = time.perf_counter()
    for _ in range(args.steps):
        totals.append(oracle_step_costs(args, Wh, system)["full_step_s"])
    wall = (time.perf_counter() - t) / args.steps
    step_s = sum(totals) / len(totals)
    v = K_STENCILS / step_s
    desc = _oracle_desc(Wh["n"], len(system[0]["colidx"]))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": v, "unit": "stencils/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": step_s * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": workload_desc(args), "precision": args.precision, "hess_mode": args.hess_mode,
                   "oracle_eval_sample": ORACLE_EVAL_SAMPLE, "measured_wall_s_per_step": wall},
        "cpu_baseline": {"value": v, "unit": "stencils/s", "cores": 1, "kind": "oracle", "sample": desc},
        "e2e": {"value": v, "unit": "stencils/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def run_per_type(args):
    """Stencil evaluation rate of each type alone (same recipe as the C1 mix, one type per launch).

    Each type gets K stencils with their own vertices; eps_x, then ``warmup`` untimed and ``steps``
    timed evaluations per precision, timed by CUDA events on the current stream.  The launches
    come in the order of ``synth.TYPE_IDS``, FP64 before mixed, which is how an instruction-count
    capture of this command is read per type."""
    import torch
    import synth
    import paper_2308_09400_gb300 as g

    torch.cuda.set_device(0)
    dev = torch.device("cuda", 0)
    k = args.per_type
    rows = {}
    for kind in synth.TYPE_IDS:
        B = synth.batch_stencils(k, mix=((kind, 1.0),))
        x = torch.tensor(B["x"], device=dev)
        st = torch.tensor(B["stencils"], device=dev)
        eps = g.compute_eps_x(x, st)
        row = {}
        for prec in ("fp64", "mixed"):
            out = None
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            for it in range(args.warmup + args.steps):
                if it == args.warmup:
                    torch.cuda.synchronize()
                    t0.record()
                out = g.eval_stencils(x, st, eps, B["dhat"], KAPPA, precision=prec, mode="blocks", out=out)
            t1.record()
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / max(args.steps, 1)
            active = int(((out["flags"] & 1) != 0).sum().item())
            row[prec] = {"ms": ms, "stencils_per_s": k / ms * 1e3, "active": active}
        rows[kind] = row
    print(json.dumps({"per_type": rows, "stencils_per_type": k, "steps": args.steps, "warmup": args.warmup,
                      "output": "energy, gradient, projected Hessian as 3x3 sub-blocks, flags"}))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.per_type > 0:
        run_per_type(args)
    else:
        run_gpu(args)


if __name__ == "__main__":
    main()
