"""Benchmark: space-time DoFs/s to relative residual 1e-8 on GB300.

Workload (default "square64"): heat equation on (0,1)^2 x (0,1), B-spline
degree 2 in space and time, 64 x 64 knot spans, 256 time slabs x 2 time
elements (4 194 304 space-time dofs), theta = 1, right-hand side from i.i.d.
N(0,1) B-spline coefficients (seed 2), zero initial guess.  Solver: FGMRES(20)
right-preconditioned by one time-multigrid V-cycle (damped block Jacobi,
omega = 1/2, nu1 = nu2 = 1, slab inverses by real-Schur time transform + fast
diagonalisation in space), to ||f - L u|| <= 1e-8 ||f||.

One step = one whole solve with the right-hand side resident in HBM.  `value`
is the mixed-precision method (FP32 V-cycle, FP64 outer residual and update);
the plain FP64 method on the same workload is reported beside it.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOADS = {
    # name: (dim, spans, degree, slabs, ne, tol, seed)
    "square64": (2, (64, 64), 2, 256, 2, 1e-8, 2),
    "square128_p3": (2, (128, 128), 3, 1024, 2, 1e-8, 3),
    "cube48_x16": (3, (48, 48, 48), 2, 128, 2, 1e-8, 400),
    "interval16": (1, (16,), 2, 8, 4, 1e-10, 1),
}
# right-hand side: "coeffs" = N(0,1) B-spline coefficients (one seed per rhs),
# "bumps" = 32 space-time Gaussian bumps; number of rhs solved together;
# FGMRES restart (memory); variants measured beside the headline
RHS = {"square64": ("coeffs", 1, 20, "all"), "square128_p3": ("bumps", 1, 20, "min"),
       "cube48_x16": ("coeffs", 16, 10, "none"), "interval16": ("coeffs", 1, 20, "all")}
METRIC = "space-time DoFs/s to rel. residual 1e-8, mixed vs FP64 plain; serve p50/p99"
UNIT = "DoFs/s"
L2_FLUSH_BYTES = 256 << 20


def reduce_max(value, device="cpu"):
    """Max over the ranks of the process group (identity without one)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_value(dofs_per_rank, world, ms_max):
    """Whole-job throughput: every rank's dofs over the slowest rank's time."""
    return dofs_per_rank * world / (ms_max / 1e3)


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


# ----------------------------------------------------------------------------
# CPU oracle leg (runs in a child process, single-threaded BLAS)
# ----------------------------------------------------------------------------

def cpu_leg(args):
    """Time the oracle's FGMRES + V-cycle solve on a bounded sample of the
    workload: the same spatial grid, degree and slab size with fewer slabs."""
    import numpy as np
    from oracle import assemble as A
    from oracle import solve as S
    from paper_1802_09277_gb300 import inputs
    d, spans, p, N, ne, tol, seed = WORKLOADS[args.workload]
    n_sample = args.sample_slabs
    pr = A.Problem(d, spans, p, ne, n_sample, theta=1.0, T=float(n_sample) / N)
    c = inputs.normal_coeffs(seed, pr.ndofs)
    f = A.load_from_coeffs(pr, c)
    H = S.Hierarchy(pr)
    L = H.levels[0].L
    reps, total, iters = 0, 0.0, 0
    t_end = time.perf_counter() + args.cpu_seconds
    while True:
        t0 = time.perf_counter()
        u, it, hist = S.fgmres(L, f, lambda v: S.vcycle(H, v), tol=tol, restart=20)
        total += time.perf_counter() - t0
        reps += 1
        iters = it
        if time.perf_counter() >= t_end or reps >= 50:
            break
    out = {"value": pr.ndofs * reps / total, "seconds_per_solve": total / reps,
           "iterations": iters, "sample_dofs": pr.ndofs, "sample_slabs": n_sample,
           "reps": reps}
    print(json.dumps(out))


def run_cpu_leg(workload, sample_slabs, seconds):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload", workload,
           "--sample-slabs", str(sample_slabs), "--cpu-seconds", str(seconds)]
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=600)
    if res.returncode != 0:
        raise RuntimeError("cpu leg failed: " + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


# ----------------------------------------------------------------------------
# clocks
# ----------------------------------------------------------------------------

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index, path=None):
        self.idx = str(gpu_index)
        self.proc = None
        self.keep = path is not None
        self.path = path or os.path.join(tempfile.gettempdir(),
                                         "st_bench_clocks_%d_%s.csv" % (os.getpid(), self.idx))

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", self.idx, "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
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
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not self.keep:
            try:
                os.remove(self.path)
            except OSError:
                pass
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# GPU arm
# ----------------------------------------------------------------------------

def gpu_arm(args, rank, world):
    import numpy as np
    import torch
    from paper_1802_09277_gb300 import inputs, st

    dev = torch.device("cuda", int(os.environ.get("LOCAL_RANK", "0")))
    torch.cuda.set_device(dev)
    stream = torch.cuda.current_stream()
    d, spans, p, N, ne, tol, seed = WORKLOADS[args.workload]
    rhs_kind, nrhs, restart, vset = RHS[args.workload]
    common = dict(ne_per_slab=ne, gmres_restart=restart, max_it=300, nrhs=nrhs)
    peaks, peak_src = load_peaks()

    def make(prec, basis, outer, fused=None, spatial="fd", variant="rschur", space_ratio=0.0):
        return st.Solver(d, p, spans, N, stream=stream.cuda_stream, precision=prec, basis=basis,
                         outer=outer, fused_vcycle=args.fused if fused is None else fused,
                         spatial_solver=spatial, variant=variant, space_ratio=space_ratio,
                         **common)

    # rank r solves its own right-hand side(s) (independent replicas)
    n1 = make_len(d, spans, p, N, ne)
    c = torch.tensor(np.concatenate([inputs.normal_coeffs(seed + 1000 * rank + q, n1)
                                     for q in range(nrhs)]), dtype=torch.float64, device=dev)
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()

    def timed_solves(solver, f, steps, warmup, profile=False):
        u = torch.zeros_like(f)
        for _ in range(warmup):
            solver.solve(f, u, tol=tol)
        times, infos = [], []
        barrier()
        torch.cuda.synchronize()
        if profile:
            solver.profile(True)
        for _ in range(steps):
            flush.fill_(1.0)  # L2 flush between timed iterations (outside the events)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = solver.solve(f, u, tol=tol)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
            infos.append(info)
        torch.cuda.synchronize()
        prof = None
        if profile:
            prof = solver.profile_read()
            solver.profile(False)
        barrier()
        return times, infos, u, prof

    def timed_make(*a, **kw):
        """Setup (host factors, uploads, allocations) timed on the host clock,
        reported apart from the solve as in Table 4's setup / solve split."""
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        sv = make(*a, **kw)
        torch.cuda.synchronize()
        return sv, 1e3 * (time.perf_counter() - t0)

    # --- mixed precision (headline) ---
    sm, setup_ms = timed_make(args.precision, args.basis, args.outer)
    f = torch.empty_like(c)
    if rhs_kind == "bumps":
        cen, wid, amp = inputs.gaussian_bumps(seed + 1000 * rank, count=32, dim=d + 1)
        sm.load_gaussians(cen, wid, amp, f)
    else:
        sm.load_coeffs(c, f)
    del c
    t0 = time.perf_counter()
    tuning = sm.autotune()  # also runs inside the first solve (opt.autotune)
    autotune_ms = 1e3 * (time.perf_counter() - t0)
    clocks = ClockSampler(dev.index, args.clocks_csv)
    clocks.start()
    t_mixed, i_mixed, u_mixed, _ = timed_solves(sm, f, args.steps, args.warmup)
    clk = clocks.stop()
    ms = sum(t_mixed) / len(t_mixed)
    # the same steps again with per-launch CUDA events (library profiling
    # hook) for the per-kernel roofline; kept out of the headline timing
    t_prof, _, _, prof = timed_solves(sm, f, args.steps, 0, profile=True)
    ms_prof = sum(t_prof) / len(t_prof)
    ms_max = reduce_max(ms, dev)

    # --- end to end through the public API with host buffers ---
    f_host = f.cpu().pin_memory()
    u_host = torch.empty_like(f_host).pin_memory()
    f_dev = torch.empty_like(f)
    u_dev = torch.zeros_like(f)
    e2e_t = []
    for k in range(args.warmup + max(2, args.steps // 2)):
        flush.fill_(1.0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        f_dev.copy_(f_host, non_blocking=True)
        sm.solve(f_dev, u_dev, tol=tol)
        u_host.copy_(u_dev, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        if k >= args.warmup:
            e2e_t.append(e0.elapsed_time(e1))
    e2e_ms = sum(e2e_t) / len(e2e_t)
    del f_host, u_host, f_dev, u_dev

    # --- the other variants on the same workload (fewer steps, no profiling) ---
    variants = {}
    u64 = None
    u_mixed = u_mixed.cpu()
    ndofs_h = sm.ndofs
    sm.close()
    torch.cuda.empty_cache()
    allv = (("fp64", "nodal", "fgmres"), ("fp64", "spectral", "fgmres"),
            ("mixed_fp32", "nodal", "fgmres"), ("mixed_fp32", "spectral", "fgmres"),
            ("mixed_fp32", "spectral", "ir"), ("mixed_tf32", "spectral", "ir"),
            ("mixed_bf16", "spectral", "ir"), ("mixed_tf32", "spectral", "fgmres"))
    allv = [v + (args.fused, "fd", "rschur", 0.0) for v in allv]
    # the inexact spatial solves (MinRes block solves inside the B-spline-basis
    # smoother) with the three factorisations of Table 4
    for fac in ("rschur", "eig", "cschur"):
        allv.append(("mixed_fp32", "nodal", "fgmres", args.fused, "minres", fac, 0.0))
    # space-time coarsening of the B-spline-basis V-cycle (space while tau/h^2 > 1)
    allv.append(("mixed_fp32", "nodal", "fgmres", args.fused, "fd", "rschur", 1.0))
    allv.append((args.precision, args.basis, args.outer, 1 - args.fused, "fd", "rschur", 0.0))
    chosen = {"all": allv, "min": [allv[0], allv[-1]], "none": []}[vset]
    for prec, basis, outer, fz, spatial, fac, sratio in chosen:
        name = "fp64_plain" if (prec, basis, spatial, sratio) == ("fp64", "nodal", "fd", 0.0) \
            else "%s_%s_%s" % (prec, basis, outer)
        if spatial != "fd":
            name += "_" + spatial + ("" if fac == "rschur" else "_" + fac)
        if sratio > 0:
            name += "_spacetime"
        if fz != args.fused:
            name += "_fused" if fz else "_levelwise"
        elif (prec, basis, outer, spatial, sratio) == (args.precision, args.basis, args.outer,
                                                       "fd", 0.0) and name != "fp64_plain":
            continue
        sv, sv_setup_ms = timed_make(prec, basis, outer, fz, spatial, fac, sratio)
        tv, iv, uv, _ = timed_solves(sv, f, max(1, args.steps // 2), 1)
        msv = sum(tv) / len(tv)
        variants[name] = {"precision": prec, "basis": basis, "outer": outer, "fused_vcycle": fz,
                          "spatial_solver": spatial, "variant": fac, "space_ratio": sratio,
                          "levels": "".join(k for _, _, k in sv.level_shapes()[1:]),
                          "setup_ms": sv_setup_ms,
                          "ms_per_step": msv,
                          "value": sv.ndofs * world / (msv / 1e3),
                          "iterations": iv[-1]["iterations"],
                          "refinements": iv[-1].get("refinements", 0),
                          "rel_residual": iv[-1]["rel_residual"]}
        if name == "fp64_plain":
            u64 = uv.cpu()
        del uv
        sv.close()
        torch.cuda.empty_cache()
    # the FP64 reference solve (skipped where one takes about a minute)
    v64 = variants.get("fp64_plain")
    ms64 = v64["ms_per_step"] if v64 else None
    i64 = [{"iterations": v64["iterations"] if v64 else None,
            "rel_residual": v64["rel_residual"] if v64 else None}]
    rel_diff = (float(torch.linalg.norm(u_mixed - u64) / torch.linalg.norm(u64))
                if u64 is not None else None)
    ndofs = ndofs_h

    # --- roofline of the dominant kernel class ---
    dom = max(prof, key=lambda k: prof[k]["ms"])
    pd = prof[dom]
    per_launch_ms = pd["ms"] / max(pd["launches"], 1)
    launches = sum(v["launches"] for v in prof.values())
    result = {
        "ndofs": ndofs, "ms_mixed": ms, "ms_mixed_max": ms_max, "ms64": ms64, "ms_prof": ms_prof,
        "iters_mixed": i_mixed[-1]["iterations"], "res_mixed": i_mixed[-1]["rel_residual"],
        "refin_mixed": i_mixed[-1].get("refinements", 0),
        "iters64": i64[-1]["iterations"], "res64": i64[-1]["rel_residual"],
        "rel_diff_mixed_vs_fp64": rel_diff, "e2e_ms": e2e_ms, "bytes_h2d": f.numel() * 8,
        "bytes_d2h": f.numel() * 8, "prof": prof, "dominant": dom,
        "per_launch_ms": per_launch_ms, "launches": launches // max(args.steps, 1),
        "launches_total": launches, "clocks": clk, "peaks": peaks, "peak_src": peak_src,
        "variants": variants, "tuning": tuning,
        "setup_ms": {"setup": setup_ms, "autotune": autotune_ms},
        "traffic_key": (args.workload, args.precision, args.basis, args.outer),
    }
    return result


def serve_arm(args):
    """Serving workload: Poisson arrivals of solve requests of mixed
    configurations through st_serve (continuous batching)."""
    import threading
    import numpy as np
    from paper_1802_09277_gb300 import inputs, st
    nreq, rate, seed = args.serve_requests, args.serve_rate, 5
    arrivals = inputs.poisson_arrivals(seed, nreq, rate)
    mix = inputs.serving_mix(seed, nreq)
    ne = 2
    reqs = []
    for i, (sp, p, N) in enumerate(mix):
        n = (sp + p - 2) ** 2 * N * (ne + p)
        reqs.append((sp, p, N, inputs.normal_coeffs(10000 + i, n)))
    srv = st.Server(workers=args.serve_workers, max_batch=8, precision=args.precision,
                    basis="spectral", outer="ir", ne_per_slab=ne, gmres_restart=20, max_it=300)
    tickets = [None] * nreq
    t0 = time.perf_counter()

    def submitter():
        for i, (sp, p, N, c) in enumerate(reqs):
            dt = t0 + arrivals[i] - time.perf_counter()
            if dt > 0:
                time.sleep(dt)
            tickets[i] = srv.submit(2, p, (sp, sp), N, c, tol=1e-8, coeffs=True)

    th = threading.Thread(target=submitter)
    th.start()
    lat, dofs, worst, batches, bad = [], 0, 0.0, [], 0
    for i in range(nreq):
        while tickets[i] is None:
            time.sleep(1e-4)
        res, u = srv.wait(tickets[i], timeout=600.0)
        if res["status"] != 0:
            bad += 1
        lat.append(res["latency_seconds"])
        dofs += res["n_dofs"]
        worst = max(worst, res["rel_residual"])
        batches.append(res["batch_size"])
    makespan = time.perf_counter() - t0
    th.join()
    srv.stop()
    lat = np.sort(np.array(lat))
    return {"requests": nreq, "arrival_rate_per_s": rate, "workers": args.serve_workers,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "throughput_dofs_per_s": dofs / makespan, "makespan_s": makespan, "total_dofs": int(dofs),
            "max_rel_residual": worst, "failed": bad, "mean_batch": float(np.mean(batches)),
            "precision": args.precision, "tol": 1e-8}


def make_len(d, spans, p, N, ne):
    nx = 1
    for s in spans:
        nx *= s + p - 2
    return N * (ne + p) * nx


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# over the class's launches in one solve, ncu with its default cache flush
# between launches) for (workload, precision, basis, outer, kernel class);
# the capture is summarised in the profiles/ file named beside it.  An entry
# is removed whenever a kernel of the class changes.
TRAFFIC = {
    ("square64", "mixed_tf32", "spectral", "ir", "spec"):
        (1.359e7, "profiles/traffic_square64_mixed_tf32_spectral_ir.md"),
}


def roofline_entry(r):
    """Roofline of the kernel class with the largest share of device time:
    achieved = algorithmic bytes (or flops) of its launches / their summed
    CUDA-event time."""
    peaks = r["peaks"]
    dom = r["dominant"]
    pd = r["prof"][dom]
    secs = pd["ms"] / 1e3
    clk_max = peaks.get("sm_max_mhz", 2070.0) * 1e6
    tr = TRAFFIC.get(r["traffic_key"] + (dom,))
    base = {"kernel": dom, "per_launch_ms": pd["ms"] / max(1, pd["launches"]),
            "launches": pd["launches"], "traffic": tr[0] if tr else None,
            "algorithmic_bytes_per_launch": pd["bytes"] / max(1, pd["launches"])}
    if tr:
        base["traffic_source"] = tr[1]
    if dom == "gemm32":  # FP32 FMA on CUDA cores: 152 SMs x 128 lanes x 2 flop x max clock
        peak = 152 * 128 * 2 * clk_max / 1e12
        ach = pd["flops"] / secs / 1e12
        base.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_note="FP32 CUDA-core FMA rate: unit counts x max SM clock")
        return base
    if dom == "stencil_df":  # double-float on the FP32 pipe: 15 FP32 instructions per 2-flop FMA
        peak = 152 * 128 * clk_max * 2 / 15 / 1e12
        ach = pd["flops"] / secs / 1e12
        base.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_note="FP32 lane rate x max SM clock x 2 flops / 15 instructions per "
                              "double-float multiply-add")
        return base
    if dom in ("stencil64", "gemm64"):  # FP64 pipe: GB300's 1.25 TFLOP/s dense FP64
        peak = 1.25
        ach = pd["flops"] / secs / 1e12
        base.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_note="GB300 FP64 rate 1.25 TFLOP/s (probe: 1.26)")
        return base
    ach = pd["bytes"] / secs / 1e9
    peak = peaks["hbm_gbs"]
    base.update(bound="hbm", achieved=ach, peak=peak, unit="GB/s", frac=ach / peak,
                peak_note="%s hbm_gbs" % r["peak_src"])
    return base


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="square64", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-leg", action="store_true")
    ap.add_argument("--sample-slabs", type=int, default=8)
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the raw nvidia-smi clock samples of the timed region in this file")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-workers", type=int, default=4)
    ap.add_argument("--basis", default="spectral", choices=["spectral", "nodal"])
    ap.add_argument("--outer", default="ir", choices=["ir", "fgmres", "mg"])
    ap.add_argument("--precision", default="mixed_tf32",
                    choices=["mixed_fp32", "mixed_tf32", "mixed_bf16", "fp64"])
    ap.add_argument("--fused", type=int, default=0, choices=[0, 1],
                    help="eigenbasis V-cycle as one shared-memory kernel (1) or level by level (0)")
    args = ap.parse_args()

    if args.cpu_leg:
        cpu_leg(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    d, spans, p, N, ne, tol, seed = WORKLOADS[args.workload]
    cfg = {"workload": args.workload, "domain": "unit %s" % {1: "interval", 2: "square", 3: "cube"}[d],
           "spans": list(spans), "degree": p, "slabs": N, "time_elements_per_slab": ne,
           "theta": 1.0, "tol": tol, "solver": "V(1,1) time multigrid, omega=0.5, FGMRES(20) restart",
           "precision": args.precision, "vcycle_basis": args.basis, "outer": args.outer,
           "fused_vcycle": args.fused,
           "rhs": "N(0,1) B-spline coefficients, seed %d" % seed, "l2": "flushed between steps"}

    if args.impl == "reference":
        if rank != 0:
            return
        ncores = os.cpu_count()
        r = run_cpu_leg(args.workload, args.sample_slabs, max(5.0, args.cpu_seconds))
        line = {"impl": "reference", "metric": METRIC, "value": r["value"], "unit": UNIT,
                "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * r["seconds_per_solve"], "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "config": cfg,
                "cpu_baseline": {"value": r["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "host_cores_available": ncores,
                                 "sample": "%d of %d slabs (%d dofs), same grid/degree/slab size, "
                                           "%d solves" % (r["sample_slabs"], N, r["sample_dofs"], r["reps"])},
                "e2e": {"value": r["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line))
        return

    if world > 1:
        import torch
        torch.distributed.init_process_group("nccl")
    r = gpu_arm(args, rank, world)
    if rank != 0:
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
        return
    ndofs = r["ndofs"]
    value = job_value(ndofs, world, r["ms_mixed_max"])
    serve = None
    if not args.no_serve and world == 1:
        try:
            serve = serve_arm(args)
        except Exception as e:
            serve = {"error": str(e)[:300]}
    cpu = None
    if not args.no_cpu and world == 1:
        try:
            cb = run_cpu_leg(args.workload, args.sample_slabs, args.cpu_seconds)
            cpu = {"value": cb["value"], "unit": UNIT, "cores": 1, "kind": "oracle",
                   "host_cores_available": os.cpu_count(),
                   "sample": "%d of %d slabs (%d dofs), same grid/degree/slab size, FGMRES + V-cycle "
                             "with sparse-LU slab solves, %d solves" % (
                                 cb["sample_slabs"], N, cb["sample_dofs"], cb["reps"])}
        except Exception as e:  # the GPU number stands without it
            cpu = {"value": None, "unit": UNIT, "cores": 1, "kind": "oracle", "error": str(e)[:200]}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_mixed_max"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": cfg,
        "iterations": r["iters_mixed"], "refinements": r["refin_mixed"],
        "rel_residual": r["res_mixed"],
        "fp64_plain": None if r["ms64"] is None else {
                       "value": ndofs * world / (r["ms64"] / 1e3), "ms_per_step": r["ms64"],
                       "iterations": r["iters64"], "rel_residual": r["res64"], "dtype": "f64",
                       "basis": "nodal"},
        "variants": r["variants"],
        "setup_ms": r["setup_ms"],
        "mixed_vs_fp64_solution_rel_diff": r["rel_diff_mixed_vs_fp64"],
        "roofline": roofline_entry(r),
        "profiled_ms_per_step": r["ms_prof"],
        "kernel_classes": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                               "share": v["ms"] / max(1e-12, sum(x["ms"] for x in r["prof"].values()))}
                           for k, v in r["prof"].items() if v["launches"]},
        "cpu_baseline": cpu,
        "serve": serve,
        "e2e": {"value": ndofs * world / (r["e2e_ms"] / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": r["bytes_h2d"], "d2h_bytes_per_step": r["bytes_d2h"]},
        "gpu_launches": r["launches"],
        "transform_autotune": [{"axis": a, "choice": ("cuda_cores" if c == 0 else
                                                       "tensor_cores_%d_cta_per_sm" % c),
                                "ms_per_pass": ms} for a, (c, ms) in enumerate(r["tuning"])],
        "clocks": r["clocks"],
    }
    print(json.dumps(line))
    if world > 1:
        import torch
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
