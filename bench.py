"""Benchmark: space-time DoFs/s to relative residual 1e-8 on GB300.

Default workload "cube48_x16": heat equation on (0,1)^3 x (0,1), B-spline
degree 2 in space and time, 48^3 knot spans, 128 time slabs x 2 time
elements (56 623 104 space-time dofs per right-hand side), theta = 1,
16 right-hand sides of i.i.d. N(0,1) B-spline coefficients (seeds 400..415)
solved together, zero initial guess, to ||f - L u|| <= 1e-8 ||f|| for every
right-hand side.  Headline method: mixed precision -- iterative refinement
with an FP64-accurate residual and FP64 update around an FP32 FGMRES(10),
right-preconditioned by one time-multigrid V(4,4) cycle (damped block
Jacobi, omega = 1/2, slab inverses by the real Schur time factors and fast
diagonalisation in space, V-cycle in the spatial eigenbasis); the spatial
transforms at the refinement boundary run as split TF32 on the tensor cores
(FP32 accuracy).  Beside it on the same workload: the plain FP64 method
(FP64 FGMRES and FP64 V-cycle) and FP64-outer FGMRES with the FP32 V-cycle.
The 2D degree-3 workload "square128_p3" (128^2 spans, 1024 slabs, 32
space-time Gaussian bumps) is measured after it with TF32 and BF16
transforms and FP64 plain.  Every result carries the FP64 oracle's residual
of the returned solution on sampled slabs.

One step = one whole solve with the right-hand sides resident in HBM.

  python bench.py [--steps K] [--warmup W] [--gpus N] [--impl reference]
                  [--workload NAME]
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
# FGMRES restart (memory: 16 FP64 rhs of cube48 are 7.25 GB per vector)
RHS = {"square64": ("coeffs", 1, 20), "square128_p3": ("bumps", 1, 20),
       "cube48_x16": ("coeffs", 16, 10), "interval16": ("coeffs", 1, 20)}
# the plain FP64 method on each workload: FP64 FGMRES + FP64 V-cycle.  On the
# large workloads its V-cycle runs in the spatial eigenbasis (the same
# iterates as the B-spline-basis cycle, whose FP64 transforms in every
# smoothing step take about a minute per cube48_x16 solve)
FP64_PLAIN = {"square64": ("fp64", "nodal", "fgmres"), "interval16": ("fp64", "nodal", "fgmres"),
              "square128_p3": ("fp64", "spectral", "fgmres"),
              "cube48_x16": ("fp64", "spectral", "fgmres")}
# variant sets measured beside the headline; extra workloads measured after it
VSET = {"square64": "all", "interval16": "all", "square128_p3": "min", "cube48_x16": "outer64"}
EXTRA = {"cube48_x16": ["square128_p3"]}
# the oracle's bounded CPU sample of each workload: spatial spans and slabs
# (same dimension, degree, time elements per slab and slab length)
ORACLE_SAMPLE = {"square64": ((64, 64), 8), "square128_p3": ((16, 16), 8),
                 "cube48_x16": ((8, 8, 8), 8), "interval16": ((16,), 8)}
METRIC = "space-time DoFs/s to rel. residual 1e-8, mixed vs FP64 plain; serve p50/p99"
# smoothing steps of every V-cycle in the bench: V(4,4), measured best or
# close to it on cube48_x16, square128_p3 and square64 (the sweeping level
# kernels make every level one pass whatever nu, so more smoothing costs
# arithmetic only and saves Krylov steps); the library default is V(1,1)
NU = (4, 4)
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


def workload_config(name, precision, basis, outer, fused):
    d, spans, p, N, ne, tol, seed = WORKLOADS[name]
    kind, nrhs, restart = RHS[name]
    if kind == "bumps":
        rhs = "32 space-time Gaussian bumps (centres U(0,1)^%d, widths U(0.05,0.2), " \
              "amplitudes N(0,1)), seed %d" % (d + 1, seed)
    elif nrhs > 1:
        rhs = "%d right-hand sides of N(0,1) B-spline coefficients, seeds %d..%d, solved " \
              "together" % (nrhs, seed, seed + nrhs - 1)
    else:
        rhs = "N(0,1) B-spline coefficients, seed %d" % seed
    if outer == "ir":
        solver = ("iterative refinement (FP64-accurate residual, FP64 update) around FP32 "
                  "FGMRES(%d), right-preconditioned by one V(%d,%d) time-multigrid cycle, "
                  "omega=0.5" % ((restart,) + NU))
    elif outer == "mg":
        solver = "multigrid iteration with V(%d,%d) time-multigrid cycles, omega=0.5" % NU
    else:
        solver = ("FP64 FGMRES(%d), right-preconditioned by one V(%d,%d) time-multigrid cycle, "
                  "omega=0.5" % ((restart,) + NU))
    return {"workload": name,
            "domain": "unit %s" % {1: "interval", 2: "square", 3: "cube"}[d],
            "spans": list(spans), "degree": p, "slabs": N, "time_elements_per_slab": ne,
            "theta": 1.0, "tol": tol, "nrhs": nrhs, "solver": solver, "precision": precision,
            "vcycle_basis": basis, "outer": outer, "fused_vcycle": fused, "rhs": rhs,
            "l2": "flushed between steps (256 MB write)"}


# ----------------------------------------------------------------------------
# CPU oracle legs (a child process with single-threaded BLAS; the all-cores
# leg runs one oracle solve per core in a spawned process pool)
# ----------------------------------------------------------------------------

_ORACLE = {}


def _oracle_init(workload):
    """Build the oracle's sample problem and multigrid hierarchy (setup,
    not timed, as in Table 4's setup / solve split)."""
    from oracle import assemble as A
    from oracle import solve as S
    d, spans, p, N, ne, tol, seed = WORKLOADS[workload]
    sspans, ns = ORACLE_SAMPLE[workload]
    pr = A.Problem(d, sspans, p, ne, ns, theta=1.0, T=float(ns) / N)
    _ORACLE.update(pr=pr, H=S.Hierarchy(pr), tol=tol, seed=seed)


def _oracle_solve(k):
    """One oracle solve (FGMRES + V-cycle with sparse-LU slab solves) of the
    sample problem with right-hand side number k; returns seconds."""
    from oracle import assemble as A
    from oracle import solve as S
    from paper_1802_09277_gb300 import inputs
    pr, H = _ORACLE["pr"], _ORACLE["H"]
    f = A.load_from_coeffs(pr, inputs.normal_coeffs(_ORACLE["seed"] + k, pr.ndofs))
    t0 = time.perf_counter()
    S.fgmres(H.levels[0].L, f, lambda v: S.vcycle(H, v, nu1=NU[0], nu2=NU[1]), tol=_ORACLE["tol"],
             restart=20)
    return time.perf_counter() - t0


def cpu_leg(args):
    """Time the oracle on the sample: `single` solves on one core for about
    `seconds`, then rounds of one solve per core on `procs` cores (a round is
    one step of the reference arm)."""
    import multiprocessing as mp
    _oracle_init(args.workload)
    pr = _ORACLE["pr"]
    out = {"sample_dofs": pr.ndofs, "sample_spans": list(pr.spans), "sample_slabs": pr.N}
    single = []
    t_end = time.perf_counter() + args.cpu_seconds
    while True:
        single.append(_oracle_solve(len(single)))
        if len(single) >= max(1, args.cpu_single_min) and time.perf_counter() >= t_end:
            break
    out["single"] = {"value": pr.ndofs / (sum(single) / len(single)),
                     "seconds_per_solve": sum(single) / len(single), "solves": len(single)}
    P = args.cpu_procs
    if P > 1:
        ctx = mp.get_context("spawn")
        with ctx.Pool(P, initializer=_oracle_init, initargs=(args.workload,)) as pool:
            pool.map(_oracle_solve, range(P))  # every worker has built its hierarchy
            rounds = []
            t_end = time.perf_counter() + args.cpu_seconds
            for k in range(args.cpu_warmup + args.cpu_rounds):
                t0 = time.perf_counter()
                pool.map(_oracle_solve, [P * k + q for q in range(P)], chunksize=1)
                dt = time.perf_counter() - t0
                if k >= args.cpu_warmup:
                    rounds.append(dt)
                if args.cpu_rounds_bounded and time.perf_counter() >= t_end and rounds:
                    break
        out["all"] = {"value": P * pr.ndofs / (sum(rounds) / len(rounds)), "cores": P,
                      "seconds_per_round": sum(rounds) / len(rounds), "rounds": len(rounds)}
    print(json.dumps(out))


def run_cpu_leg(workload, seconds, procs, rounds=1000, warmup=0, bounded=True, single_min=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, os.path.abspath(__file__), "--cpu-leg", "--workload", workload,
           "--cpu-seconds", str(seconds), "--cpu-procs", str(procs), "--cpu-rounds", str(rounds),
           "--cpu-warmup", str(warmup), "--cpu-single-min", str(single_min)]
    if bounded:
        cmd.append("--cpu-rounds-bounded")
    res = subprocess.run(cmd, capture_output=True, text=True, env=env, timeout=1800)
    if res.returncode != 0:
        raise RuntimeError("cpu leg failed: " + res.stderr[-2000:])
    return json.loads(res.stdout.strip().splitlines()[-1])


def sample_text(workload, r):
    d, spans, p, N, ne, tol, seed = WORKLOADS[workload]
    return ("oracle FGMRES(20) + V(%d,%d) with sparse-LU slab solves on a sample of %s: %s spans, "
            "%d of %d slabs (%d dofs), same degree, time elements and slab length; "
            "N(0,1) coefficient rhs; setup (LU factorisations) not timed" % (
                NU[0], NU[1], workload, "x".join(str(s) for s in r["sample_spans"]),
                r["sample_slabs"], N, r["sample_dofs"]))


# ----------------------------------------------------------------------------
# FP64 oracle residual of a returned solution on sampled slabs
# ----------------------------------------------------------------------------

def oracle_slab_residual(workload, sols, cache, rank=0, slabs_per_rhs=6):
    """||f_n - A u_n + B u_{n-1}|| / ||f_n|| summed over sampled slabs n of
    the first and last right-hand side, with A, B and f_n from the FP64 oracle
    (slab blocks of Eq. 2.4-2.5, the exact load vector).  sols: {name: host
    float64 array of all right-hand sides}; returns {name: relative residual}."""
    import numpy as np
    from oracle import assemble as A
    from paper_1802_09277_gb300 import inputs
    d, spans, p, N, ne, tol, seed = WORKLOADS[workload]
    kind, nrhs, _ = RHS[workload]
    pr = A.Problem(d, spans, p, ne, N, theta=1.0)
    m = pr.Nt * pr.Nx
    picks = sorted({0, 1, N // 2, N - 1} | {int(x) for x in np.random.default_rng(7).integers(
        2, N - 1, max(0, slabs_per_rhs - 4))})
    rhs_ids = sorted({0, nrhs - 1})
    if "blocks" not in cache:
        cache["blocks"] = A.slab_blocks(pr)
        F = {}
        if kind == "bumps":
            cen, wid, amp = inputs.gaussian_bumps(seed + 1000 * rank, count=32, dim=d + 1)
            Fs = A.bumps_load(pr, cen, wid, amp, slabs=picks).reshape(len(picks), m)
            for i, n in enumerate(picks):
                F[(0, n)] = Fs[i]
        else:
            # all slabs are alike, so a problem of len(picks) slabs holds the
            # picked slabs' loads (M_t (x) M_x) c_n
            sub = A.Problem(d, spans, p, ne, len(picks) * len(rhs_ids), theta=1.0,
                            T=float(len(picks) * len(rhs_ids)) / N)
            cs = []
            for q in rhs_ids:
                c = inputs.normal_coeffs(seed + 1000 * rank + q, N * m).reshape(N, m)
                cs += [c[n] for n in picks]
            Fs = A.load_from_coeffs(sub, np.concatenate(cs)).reshape(-1, m)
            i = 0
            for q in rhs_ids:
                for n in picks:
                    F[(q, n)] = Fs[i]
                    i += 1
        cache["F"] = F
    Ab, Bb = cache["blocks"]
    out = {}
    for name, u in sols.items():
        U = np.asarray(u).reshape(nrhs, N, m)
        num = den = 0.0
        for (q, n), f in cache["F"].items():
            r = f - Ab @ U[q, n] + (Bb @ U[q, n - 1] if n else 0.0)
            num += float(r @ r)
            den += float(f @ f)
        out[name] = float(np.sqrt(num / den))
    out["_sampled"] = "slabs %s of rhs %s" % (picks, rhs_ids)
    return out


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
    wl = args.workload
    d, spans, p, N, ne, tol, seed = WORKLOADS[wl]
    rhs_kind, nrhs, restart = RHS[wl]
    common = dict(ne_per_slab=ne, gmres_restart=restart, max_it=300, nrhs=nrhs, nu1=NU[0],
                  nu2=NU[1])
    peaks, peak_src = load_peaks()

    def make(prec, basis, outer, fused=None, spatial="fd", variant="rschur", space_ratio=0.0,
             rhs_per_handle=None):
        kw = dict(common)
        if rhs_per_handle:
            kw["nrhs"] = rhs_per_handle
        return st.Solver(d, p, spans, N, stream=stream.cuda_stream, precision=prec, basis=basis,
                         outer=outer, fused_vcycle=args.fused if fused is None else fused,
                         spatial_solver=spatial, variant=variant, space_ratio=space_ratio,
                         **kw)

    # rank r solves its own right-hand side(s) (independent replicas)
    n1 = make_len(d, spans, p, N, ne)
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
    f = torch.empty(nrhs * n1, dtype=torch.float64, device=dev)
    if rhs_kind == "bumps":
        cen, wid, amp = inputs.gaussian_bumps(seed + 1000 * rank, count=32, dim=d + 1)
        sm.load_gaussians(cen, wid, amp, f)
    else:
        c = torch.tensor(np.concatenate([inputs.normal_coeffs(seed + 1000 * rank + q, n1)
                                         for q in range(nrhs)]), dtype=torch.float64, device=dev)
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
    # st_solve_host streams the workload's right-hand sides in batches of
    # e2e_batch systems: each batch's copies overlap its neighbours' solves
    e2e_batch = args.e2e_batch if nrhs % max(1, args.e2e_batch) == 0 else nrhs
    se, _ = timed_make(args.precision, args.basis, args.outer, rhs_per_handle=e2e_batch)
    se.autotune()
    e2e_t, e2e_iters = [], []
    for k in range(args.warmup + max(2, args.steps // 2)):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        info = se.solve_host(f_host, u_host, tol=tol)
        t1 = time.perf_counter()
        if k >= args.warmup:
            e2e_t.append(1e3 * (t1 - t0))
            e2e_iters.append(info["iterations"])
    se.close()
    del se
    e2e_ms = sum(e2e_t) / len(e2e_t)
    e2e_max_relres = info["rel_residual"]
    ud = u_host.to(dev)
    e2e_vs_resident = float(torch.linalg.vector_norm(ud - u_mixed) / torch.linalg.vector_norm(u_mixed))
    del ud
    # the same through st_solve on the full handle with the copies in series,
    # for the breakdown (CUDA events on the stream)
    f_dev = torch.empty_like(f)
    u_dev = torch.zeros_like(f)
    e2e_parts = []
    for k in range(1 + 2):
        flush.fill_(1.0)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        ev[0].record(stream)
        f_dev.copy_(f_host, non_blocking=True)
        ev[1].record(stream)
        sm.solve(f_dev, u_dev, tol=tol)
        ev[2].record(stream)
        u_host.copy_(u_dev, non_blocking=True)
        ev[3].record(stream)
        ev[3].synchronize()
        if k >= 1:
            e2e_parts.append([ev[0].elapsed_time(ev[1]), ev[1].elapsed_time(ev[2]),
                              ev[2].elapsed_time(ev[3])])
    serial = {"h2d_ms": sum(p[0] for p in e2e_parts) / len(e2e_parts),
              "solve_ms": sum(p[1] for p in e2e_parts) / len(e2e_parts),
              "d2h_ms": sum(p[2] for p in e2e_parts) / len(e2e_parts)}
    serial["total_ms"] = serial["h2d_ms"] + serial["solve_ms"] + serial["d2h_ms"]
    e2e_breakdown = {"call": "st_solve_host", "ms": e2e_ms, "rhs_per_batch": e2e_batch,
                     "batches": nrhs // e2e_batch, "iterations": max(e2e_iters),
                     "max_rel_residual": e2e_max_relres,
                     "rel_diff_vs_resident_solution": e2e_vs_resident,
                     "pinned": bool(f_host.is_pinned() and u_host.is_pinned()),
                     "timer": "host clock around the call (it returns after the last copy)",
                     "serial_st_solve": serial}
    del f_host, u_host, f_dev, u_dev

    # --- the other variants on the same workload (fewer steps, no profiling) ---
    variants = {}
    sols = {"mixed": u_mixed.cpu().numpy()}
    del u_mixed
    ndofs = sm.ndofs
    sm.close()
    torch.cuda.empty_cache()
    plain = FP64_PLAIN[wl] + (args.fused, "fd", "rschur", 0.0)
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
    chosen = {"all": allv, "min": [allv[6]],
              # FP64-outer FGMRES with the FP32 V-cycle (FP32 transforms)
              "outer64": [("mixed_fp32", "spectral", "fgmres", args.fused, "fd", "rschur", 0.0)],
              "none": []}[VSET[wl]]
    chosen = [plain] + [v for v in chosen if v != plain]
    for prec, basis, outer, fz, spatial, fac, sratio in chosen:
        is_plain = (prec, basis, outer, fz, spatial, fac, sratio) == plain
        name = "fp64_plain" if is_plain else "%s_%s_%s" % (prec, basis, outer)
        if spatial != "fd":
            name += "_" + spatial + ("" if fac == "rschur" else "_" + fac)
        if sratio > 0:
            name += "_spacetime"
        if fz != args.fused:
            name += "_fused" if fz else "_levelwise"
        elif (prec, basis, outer, spatial, sratio) == (args.precision, args.basis, args.outer,
                                                       "fd", 0.0) and not is_plain:
            continue
        sv, sv_setup_ms = timed_make(prec, basis, outer, fz, spatial, fac, sratio)
        tv, iv, uv, _ = timed_solves(sv, f, max(1, args.steps // 2), 1)
        msv = sum(tv) / len(tv)
        variants[name] = {"precision": prec, "basis": basis, "outer": outer, "fused_vcycle": fz,
                          "spatial_solver": spatial, "variant": fac, "space_ratio": sratio,
                          "levels": "".join(k for _, _, k in sv.level_shapes()[1:]),
                          "setup_ms": sv_setup_ms,
                          "ms_per_step": msv, "steps": len(tv),
                          "value": sv.ndofs * world / (msv / 1e3),
                          "iterations": iv[-1]["iterations"],
                          "refinements": iv[-1].get("refinements", 0),
                          "rel_residual": iv[-1]["rel_residual"]}
        if is_plain or VSET[wl] == "outer64":
            sols[name] = uv.cpu().numpy()
        del uv
        sv.close()
        torch.cuda.empty_cache()
    del f, flush
    torch.cuda.empty_cache()
    v64 = variants.pop("fp64_plain")
    rel_diff = float(np.linalg.norm(sols["mixed"] - sols["fp64_plain"]) /
                     np.linalg.norm(sols["fp64_plain"]))

    # --- the FP64 oracle's residual of each returned solution ---
    oracle = None
    if rank == 0 and not args.no_oracle_check:
        t0 = time.perf_counter()
        oracle = oracle_slab_residual(wl, sols, {}, rank)
        oracle["_seconds"] = time.perf_counter() - t0
    del sols

    # --- roofline of the dominant kernel class ---
    dom = max(prof, key=lambda k: prof[k]["ms"])
    pd = prof[dom]
    per_launch_ms = pd["ms"] / max(pd["launches"], 1)
    launches = sum(v["launches"] for v in prof.values())
    result = {
        "ndofs": ndofs, "ms_mixed": ms, "ms_mixed_max": ms_max, "ms_prof": ms_prof,
        "iters_mixed": i_mixed[-1]["iterations"], "res_mixed": i_mixed[-1]["rel_residual"],
        "refin_mixed": i_mixed[-1].get("refinements", 0), "fp64_plain": v64,
        "rel_diff_mixed_vs_fp64": rel_diff, "e2e_ms": e2e_ms, "e2e_breakdown": e2e_breakdown,
        "bytes_h2d": ndofs * 8,
        "bytes_d2h": ndofs * 8, "prof": prof, "dominant": dom,
        "per_launch_ms": per_launch_ms, "launches": launches // max(args.steps, 1),
        "launches_total": launches, "clocks": clk, "peaks": peaks, "peak_src": peak_src,
        "variants": variants, "tuning": tuning, "oracle": oracle,
        "setup_ms": {"setup": setup_ms, "autotune": autotune_ms},
        "traffic_key": (wl, args.precision, args.basis, args.outer),
    }
    return result


def extra_workload(args, name):
    """A second workload measured after the headline (one GPU): the mixed
    TF32 and BF16 refinement solves and the plain FP64 method, each with the
    FP64 oracle's residual of its solution on sampled slabs."""
    import torch
    from paper_1802_09277_gb300 import inputs, st
    d, spans, p, N, ne, tol, seed = WORKLOADS[name]
    rhs_kind, nrhs, restart = RHS[name]
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    specs = [("mixed_tf32", "spectral", "ir"), ("mixed_bf16", "spectral", "ir"), FP64_PLAIN[name]]
    out, sols, f = {}, {}, None
    for prec, basis, outer in specs:
        key = "fp64_plain" if (prec, basis, outer) == FP64_PLAIN[name] else "%s_%s_%s" % (
            prec, basis, outer)
        t0 = time.perf_counter()
        sv = st.Solver(d, p, spans, N, stream=stream.cuda_stream, precision=prec, basis=basis,
                       outer=outer, ne_per_slab=ne, gmres_restart=restart, max_it=300, nrhs=nrhs,
                       nu1=NU[0], nu2=NU[1])
        setup_ms = 1e3 * (time.perf_counter() - t0)
        if f is None:
            f = torch.empty(sv.ndofs, dtype=torch.float64, device="cuda")
            if rhs_kind == "bumps":
                cen, wid, amp = inputs.gaussian_bumps(seed, count=32, dim=d + 1)
                sv.load_gaussians(cen, wid, amp, f)
            else:
                import numpy as np
                c = torch.tensor(np.concatenate([inputs.normal_coeffs(seed + q, sv.ndofs // nrhs)
                                                 for q in range(nrhs)]), device="cuda")
                sv.load_coeffs(c, f)
                del c
        u = torch.zeros_like(f)
        steps = args.steps if prec != "fp64" else max(1, args.steps // 2)
        for _ in range(1 if prec == "fp64" else args.warmup):
            sv.solve(f, u, tol=tol)
        times = []
        for _ in range(steps):
            flush.fill_(1.0)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            info = sv.solve(f, u, tol=tol)
            e1.record(stream)
            e1.synchronize()
            times.append(e0.elapsed_time(e1))
        ms = sum(times) / len(times)
        out[key] = {"precision": prec, "basis": basis, "outer": outer, "setup_ms": setup_ms,
                    "ms_per_step": ms, "steps": steps, "value": sv.ndofs / (ms / 1e3),
                    "iterations": info["iterations"], "refinements": info.get("refinements", 0),
                    "rel_residual": info["rel_residual"]}
        sols[key] = u.cpu().numpy()
        del u
        sv.close()
        torch.cuda.empty_cache()
    del f, flush
    torch.cuda.empty_cache()
    if not args.no_oracle_check:
        orc = oracle_slab_residual(name, sols, {})
        for k in out:
            out[k]["oracle_rel_residual"] = orc[k]
        out["oracle_sampled"] = orc["_sampled"]
    out["config"] = workload_config(name, "mixed_tf32", "spectral", "ir", 0)
    return out


def serve_arm(args):
    """Serving workload: arrivals of solve requests of mixed configurations
    through st_serve (continuous batching).  Three runs on one server: the
    Poisson arrivals with an empty setup cache (the headline p50 / p99), the
    same arrivals again (setups cached), and a burst: the whole mix queued
    while the server is paused, then released (a deep queue, where batches of
    equal configurations form; its clock, latencies included, starts at the
    release)."""
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
    def server(group_members):
        return st.Server(workers=args.serve_workers, max_batch=8, precision=args.precision,
                         basis="spectral", outer="ir", ne_per_slab=ne, gmres_restart=20,
                         max_it=300, nu1=NU[0], nu2=NU[1], group_members=group_members)

    srv = server(args.serve_group_members)

    def run(times, burst=False):
        tickets = [None] * nreq
        t_sub = np.zeros(nreq)
        if burst:  # queue the whole mix, then let the workers batch from it
            srv.pause()
            for i, (sp, p, N, c) in enumerate(reqs):
                t_sub[i] = time.perf_counter()
                tickets[i] = srv.submit(2, p, (sp, sp), N, c, tol=1e-8, coeffs=True)
            times = np.zeros(0)
            srv.resume()
        t0 = time.perf_counter()

        def submitter():
            for i, (sp, p, N, c) in enumerate(reqs[:len(times)]):
                dt = t0 + times[i] - time.perf_counter()
                if dt > 0:
                    time.sleep(dt)
                tickets[i] = srv.submit(2, p, (sp, sp), N, c, tol=1e-8, coeffs=True)

        th = threading.Thread(target=submitter)
        th.start()
        lat, dofs, worst, batches, bad = [], 0, 0.0, [], 0
        groups, syncs_pr, launches_pr = [], [], []
        for i in range(nreq):
            while tickets[i] is None:
                time.sleep(1e-4)
            res, u = srv.wait(tickets[i], timeout=600.0)
            if res["status"] != 0:
                bad += 1
            # submission -> solution; a burst's clock starts at the release
            lat.append(res["latency_seconds"] - (max(0.0, t0 - t_sub[i]) if burst else 0.0))
            dofs += res["n_dofs"]
            worst = max(worst, res["rel_residual"])
            batches.append(res["batch_size"])
            gq = max(1, res["group_requests"])
            groups.append(gq)
            syncs_pr.append(res["host_syncs"] / gq)  # the call's share per request
            launches_pr.append(res["vector_launches"] / gq)
        makespan = time.perf_counter() - t0
        th.join()
        lat = np.sort(np.array(lat))
        return {"p50_latency_s": float(np.percentile(lat, 50)),
                "p99_latency_s": float(np.percentile(lat, 99)),
                "throughput_dofs_per_s": dofs / makespan, "makespan_s": makespan,
                "total_dofs": int(dofs), "max_rel_residual": worst, "failed": bad,
                "mean_batch": float(np.mean(batches)),
                "mean_group_requests": float(np.mean(groups)),
                "host_syncs_per_request": float(np.mean(syncs_pr)),
                "krylov_vector_launches_per_request": float(np.mean(launches_pr))}

    first = run(arrivals)
    again = run(arrivals)
    run(None, burst=True)  # fills the setup cache with the burst's batch sizes
    burst = run(None, burst=True)
    srv.stop()
    # the same burst with every configuration's batch solved alone (a second
    # server; its first burst fills its setup cache)
    srv = server(1)
    run(None, burst=True)
    alone = run(None, burst=True)
    srv.stop()
    out = {"requests": nreq, "arrival_rate_per_s": rate, "workers": args.serve_workers,
           "group_members": args.serve_group_members,
           "precision": args.precision, "tol": 1e-8, "setup_cache": "empty at start"}
    out.update(first)
    out["repeat_setups_cached"] = again
    out["burst_all_at_once_setups_cached"] = burst
    out["burst_groups_off_setups_cached"] = alone
    return out


def make_len(d, spans, p, N, ne):
    nx = 1
    for s in spans:
        nx *= s + p - 2
    return N * (ne + p) * nx


# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum, mean
# over the class's launches in one solve, ncu with its default cache flush
# between launches) for (workload, precision, basis, outer, kernel class);
# the capture is summarised in the profiles/ file named beside it.  An entry
# is removed whenever a kernel of the class changes: the double-float
# residual's (profiles/traffic_cube48_stencil_dfloat_and_sweep.md, one of the
# 16 right-hand sides scaled by 16) went when its CTAs began to cover several
# slabs, and no capture of the new kernel has been taken.
TRAFFIC = {}


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
    if dom == "stencil_df":  # double-float on the FP32 pipe: 12 FP32 instructions per 2-flop term
        peak = 152 * 128 * clk_max * 2 / 12 / 1e12
        ach = pd["flops"] / secs / 1e12
        base.update(bound="alu", achieved=ach, peak=peak, unit="TFLOP/s", frac=ach / peak,
                    peak_note="FP32 lane rate (152 SMs x 128 lanes) x max SM clock x 2 flops / "
                              "12 FP32 instructions per compensated (Dot2) double-float term")
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


# ----------------------------------------------------------------------------
# One library operation on a chosen problem (for profilers: ncu launch lists
# and section captures); prints the mean CUDA-event time per call, no bench line
# ----------------------------------------------------------------------------

def case_mode(args):
    """--case: run one operation (apply: FP64 operator; smooth: one damped
    block-Jacobi step in the handle's precision; vcycle; solve to --case-tol;
    table3: Table 3's experiment on this grid -- MinRes steps to reduce
    ||r||_{P^-1} by --case-tol for every 2x2 block of the standardised real
    Schur form of the level-0 time pencil and for its complex shifts) on
    seeded synthetic vectors."""
    import torch
    from paper_1802_09277_gb300 import inputs, st
    if args.case_op == "table3":
        import numpy as np
        s = st.Solver(args.case_dim, args.case_degree, args.case_spans, args.case_slabs,
                      ne_per_slab=args.case_ne, theta=args.case_theta, spatial_solver="minres")
        Z = s.time_factors(0)["Z"]
        m = int(np.prod(s.nx))
        f = torch.tensor(inputs.uniform_vector(5, 2 * m), dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        steps = {"rschur": 0, "complex": 0}
        i = 0
        while i < s.nt:
            if i + 1 < s.nt and Z[i + 1, i] != 0.0:
                a, b1, b2 = Z[i, i], Z[i, i + 1], Z[i + 1, i]
                w = float(np.sqrt(abs(b1 * b2)))
                for key, (c1, c2) in (("rschur", (b1, b2)), ("complex", (-w, w))):
                    its, _, _ = s.block_minres(a, c1, c2, f, u, tol=args.case_tol)
                    steps[key] = max(steps[key], int(its[0]))
                i += 2
            else:
                i += 1
        print("table3 dim=%d spans=%s p=%d nt=%d theta=%g tol=%g max_steps_rschur=%d "
              "max_steps_complex=%d" % (args.case_dim, args.case_spans, args.case_degree, s.nt,
                                        args.case_theta, args.case_tol, steps["rschur"],
                                        steps["complex"]))
        s.close()
        return
    s = st.Solver(args.case_dim, args.case_degree, args.case_spans, args.case_slabs,
                  ne_per_slab=args.case_ne, precision=args.precision, basis=args.basis,
                  outer=args.outer, fused_vcycle=args.fused,
                  spatial_solver=args.case_spatial_solver, minres_tol=args.case_minres_tol,
                  theta=args.case_theta, space_ratio=args.case_space_ratio,
                  nrhs=args.case_nrhs, nu1=args.case_nu[0], nu2=args.case_nu[1],
                  inner_tol=args.case_inner_tol, gmres_restart=args.case_restart,
                  autotune=args.case_autotune)
    n = s.ndofs
    x = torch.tensor(inputs.uniform_vector(1, n), dtype=torch.float64, device="cuda")
    f = torch.tensor(inputs.uniform_vector(2, n), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = []
    for _ in range(args.case_reps):
        ev[0].record()
        if args.case_op == "apply":
            s.apply(x, y)
        elif args.case_op == "smooth":
            s.smooth(x, f, 1)
        elif args.case_op == "vcycle":
            s.vcycle(x, f)
        else:
            s.solve(f, y, tol=args.case_tol)
        ev[1].record()
        ev[1].synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    extra = ""
    if args.case_op == "solve":
        u = torch.zeros_like(f)
        if args.case_profile:
            s.profile(True)
        info = s.solve(f, u, tol=args.case_tol)
        if args.case_profile:
            prof = s.profile_read()
            s.profile(False)
            for k, v in prof.items():
                if v["launches"]:
                    print("class=%s launches=%d ms=%.4f GB/s=%.1f" % (
                        k, v["launches"], v["ms"], v["bytes"] / max(v["ms"], 1e-9) / 1e6))
        levels = "".join(k for _, _, k in s.level_shapes()[1:])
        extra = " iterations=%d levels=%s min_ms=%.4f" % (info["iterations"], levels, min(times))
    print("op=%s dofs=%d precision=%s mean_ms=%.4f%s" % (args.case_op, n, args.precision,
                                                        sum(times) / len(times), extra))
    s.close()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="native", choices=["native", "reference"])
    ap.add_argument("--workload", default="cube48_x16", choices=sorted(WORKLOADS))
    ap.add_argument("--cpu-leg", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--cpu-procs", type=int, default=0, help="0 = every host core")
    ap.add_argument("--cpu-rounds", type=int, default=1000)
    ap.add_argument("--cpu-warmup", type=int, default=0)
    ap.add_argument("--cpu-rounds-bounded", action="store_true")
    ap.add_argument("--cpu-single-min", type=int, default=1)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--e2e-batch", type=int, default=4,
                    help="right-hand sides per batch of the end-to-end stream (st_solve_host)")
    ap.add_argument("--no-oracle-check", action="store_true")
    ap.add_argument("--clocks-csv", default=None,
                    help="keep the raw nvidia-smi clock samples of the timed region in this file")
    ap.add_argument("--serve-requests", type=int, default=512)
    ap.add_argument("--serve-rate", type=float, default=200.0)
    ap.add_argument("--serve-workers", type=int, default=8)
    ap.add_argument("--serve-group-members", type=int, default=8,
                    help="configurations per group solve call (1 = each batch alone)")
    ap.add_argument("--basis", default="spectral", choices=["spectral", "nodal"])
    ap.add_argument("--outer", default="ir", choices=["ir", "fgmres", "mg"])
    ap.add_argument("--precision", default="mixed_tf32",
                    choices=["mixed_fp32", "mixed_tf32", "mixed_bf16", "fp64"])
    ap.add_argument("--fused", type=int, default=0, choices=[0, 1],
                    help="eigenbasis V-cycle as one shared-memory kernel (1) or level by level (0)")
    # --case: one library operation on a chosen problem (profiling driver)
    ap.add_argument("--case", action="store_true")
    ap.add_argument("--case-op", default="solve",
                    choices=["apply", "smooth", "vcycle", "solve", "table3"])
    ap.add_argument("--case-dim", type=int, default=2)
    ap.add_argument("--case-spans", type=int, nargs="+", default=[64, 64])
    ap.add_argument("--case-degree", type=int, default=2)
    ap.add_argument("--case-slabs", type=int, default=256)
    ap.add_argument("--case-ne", type=int, default=2)
    ap.add_argument("--case-nrhs", type=int, default=1)
    ap.add_argument("--case-reps", type=int, default=2)
    ap.add_argument("--case-tol", type=float, default=1e-8)
    ap.add_argument("--case-theta", type=float, default=1.0)
    ap.add_argument("--case-space-ratio", type=float, default=0.0)
    ap.add_argument("--case-spatial-solver", default="fd", choices=["fd", "minres"])
    ap.add_argument("--case-minres-tol", type=float, default=1e-4)
    ap.add_argument("--case-nu", type=int, nargs=2, default=[1, 1], help="nu1 nu2")
    ap.add_argument("--case-inner-tol", type=float, default=1e-4)
    ap.add_argument("--case-restart", type=int, default=20, help="FGMRES restart (memory)")
    ap.add_argument("--case-autotune", type=int, default=1, choices=[0, 1])
    ap.add_argument("--case-profile", action="store_true",
                    help="print per-kernel-class CUDA-event times of one more solve")
    args = ap.parse_args()
    ncores = os.cpu_count() or 1
    if args.case:
        case_mode(args)
        return
    if args.cpu_procs <= 0:
        args.cpu_procs = ncores

    if args.cpu_leg:
        cpu_leg(args)
        return

    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    wl = args.workload
    cfg = workload_config(wl, args.precision, args.basis, args.outer, args.fused)

    if args.impl == "reference":
        if rank != 0:
            return
        # one step = one round of concurrent oracle solves of the sample, one
        # per host core (setup excluded); a few single-core solves beside it
        r = run_cpu_leg(wl, 0.0, args.cpu_procs, rounds=args.steps, warmup=args.warmup,
                        bounded=False, single_min=3)
        leg = r.get("all") or {"value": r["single"]["value"], "cores": 1,
                               "seconds_per_round": r["single"]["seconds_per_solve"],
                               "rounds": r["single"]["solves"]}
        cfg_ref = {k: v for k, v in cfg.items()
                   if k not in ("vcycle_basis", "outer", "fused_vcycle", "l2")}
        cfg_ref.update(precision="fp64", solver="oracle: FGMRES(20) + V(%d,%d) time multigrid "
                       "with sparse-LU slab solves (FP64, CPU)" % NU)
        line = {"impl": "reference", "metric": METRIC, "value": leg["value"], "unit": UNIT,
                "n_gpus": args.gpus, "steps": leg["rounds"], "warmup": args.warmup,
                "ms_per_step": 1e3 * leg["seconds_per_round"],
                "step": "one round of %d concurrent oracle solves of the sample, one per host "
                        "core" % leg["cores"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": cfg_ref,
                "cpu_baseline": {"value": leg["value"], "unit": UNIT, "cores": leg["cores"],
                                 "kind": "oracle", "host_cores_available": ncores,
                                 "sample": sample_text(wl, r),
                                 "single_core": {"value": r["single"]["value"], "cores": 1,
                                                 "ms_per_solve": 1e3 * r["single"]["seconds_per_solve"],
                                                 "solves": r["single"]["solves"]}},
                "e2e": {"value": leg["value"], "unit": UNIT, "h2d_bytes_per_step": 0,
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
    extra = {}
    if not args.no_extra and world == 1:
        for name in EXTRA.get(wl, []):
            try:
                extra[name] = extra_workload(args, name)
            except Exception as e:
                extra[name] = {"error": str(e)[:300]}
    serve = None
    if not args.no_serve and world == 1:
        try:
            serve = serve_arm(args)
        except Exception as e:
            serve = {"error": str(e)[:300]}
    cpu = None
    if not args.no_cpu and world == 1:
        try:
            cb = run_cpu_leg(wl, args.cpu_seconds, args.cpu_procs, bounded=True, single_min=2)
            leg = cb.get("all") or {"value": cb["single"]["value"], "cores": 1}
            cpu = {"value": leg["value"], "unit": UNIT, "cores": leg["cores"], "kind": "oracle",
                   "host_cores_available": ncores, "sample": sample_text(wl, cb),
                   "single_core": {"value": cb["single"]["value"], "cores": 1,
                                   "ms_per_solve": 1e3 * cb["single"]["seconds_per_solve"]}}
        except Exception as e:  # the GPU number stands without it
            cpu = {"value": None, "unit": UNIT, "cores": args.cpu_procs, "kind": "oracle",
                   "error": str(e)[:200]}
    v64 = r["fp64_plain"]
    orc = r["oracle"] or {}
    if v64 is not None:
        v64 = dict(v64, dtype="f64", oracle_rel_residual=orc.get("fp64_plain"))
    for k, v in r["variants"].items():
        if k in orc:
            v["oracle_rel_residual"] = orc[k]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": r["ms_mixed_max"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if args.precision == "fp64" else "f32+f64", "data": "synthetic",
        "config": cfg,
        "iterations": r["iters_mixed"], "refinements": r["refin_mixed"],
        "rel_residual": r["res_mixed"],
        "oracle_rel_residual": orc.get("mixed"),
        "oracle_check": None if not orc else {
            "what": "FP64 oracle residual ||f_n - A u_n + B u_{n-1}|| / ||f_n|| of the returned "
                    "solution (Eq. 2.4-2.5 slab blocks, exact load vector)",
            "sampled": orc.get("_sampled"), "seconds": orc.get("_seconds")},
        "fp64_plain": v64,
        "mixed_vs_fp64_speedup": (v64["ms_per_step"] / r["ms_mixed"]) if v64 else None,
        "mixed_vs_fp64_solution_rel_diff": r["rel_diff_mixed_vs_fp64"],
        "variants": r["variants"],
        "extra_workloads": extra,
        "setup_ms": r["setup_ms"],
        "roofline": roofline_entry(r),
        "profiled_ms_per_step": r["ms_prof"],
        "kernel_classes": {k: {"launches": v["launches"], "ms": round(v["ms"], 4),
                               "share": v["ms"] / max(1e-12, sum(x["ms"] for x in r["prof"].values()))}
                           for k, v in r["prof"].items() if v["launches"]},
        "cpu_baseline": cpu,
        "serve": serve,
        "e2e": {"value": ndofs * world / (r["e2e_ms"] / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": r["bytes_h2d"], "d2h_bytes_per_step": r["bytes_d2h"],
                "breakdown": r["e2e_breakdown"]},
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
