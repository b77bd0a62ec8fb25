"""Run one library operation on a chosen problem, e.g. under ncu:

  python paper_1802_09277_gb300/profile_case.py --dim 2 --spans 128 128 \
      --degree 3 --slabs 512 --precision mixed_fp32 --op smooth --reps 2

Operations: apply (FP64 operator), smooth (one damped block-Jacobi step in
the handle's precision), vcycle, solve (to --tol), table3 (Table 3's
experiment on this grid: MinRes steps to reduce ||r||_{P^{-1}} by --tol for
every 2x2 block of the standardised real Schur form of the level-0 time
pencil and for its complex shifts, st_block_minres).  Inputs are seeded
synthetic vectors; the script prints the mean CUDA-event time per call.
"""
import argparse
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(HERE))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--dim", type=int, default=2)
    ap.add_argument("--spans", type=int, nargs="+", default=[128, 128])
    ap.add_argument("--degree", type=int, default=3)
    ap.add_argument("--slabs", type=int, default=512)
    ap.add_argument("--ne", type=int, default=2)
    ap.add_argument("--precision", default="mixed_fp32")
    ap.add_argument("--op", default="smooth",
                    choices=["apply", "smooth", "vcycle", "solve", "table3"])
    ap.add_argument("--reps", type=int, default=2)
    ap.add_argument("--tol", type=float, default=1e-8)
    ap.add_argument("--basis", default="nodal", choices=["nodal", "spectral"])
    ap.add_argument("--outer", default="fgmres", choices=["fgmres", "mg", "ir"])
    ap.add_argument("--fused", type=int, default=0, choices=[0, 1])
    ap.add_argument("--spatial-solver", default="fd", choices=["fd", "minres"])
    ap.add_argument("--minres-tol", type=float, default=1e-4)
    ap.add_argument("--theta", type=float, default=1.0)
    ap.add_argument("--space-ratio", type=float, default=0.0)
    args = ap.parse_args()

    import torch
    from paper_1802_09277_gb300 import inputs, st

    if args.op == "table3":
        table3(args, st, inputs, torch)
        return
    s = st.Solver(args.dim, args.degree, args.spans, args.slabs, ne_per_slab=args.ne,
                  precision=args.precision, basis=args.basis, outer=args.outer,
                  fused_vcycle=args.fused, spatial_solver=args.spatial_solver,
                  minres_tol=args.minres_tol, theta=args.theta, space_ratio=args.space_ratio)
    n = s.ndofs
    x = torch.tensor(inputs.uniform_vector(1, n), dtype=torch.float64, device="cuda")
    f = torch.tensor(inputs.uniform_vector(2, n), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    times = []
    for _ in range(args.reps):
        ev[0].record()
        if args.op == "apply":
            s.apply(x, y)
        elif args.op == "smooth":
            s.smooth(x, f, 1)
        elif args.op == "vcycle":
            s.vcycle(x, f)
        else:
            s.solve(f, y, tol=args.tol)
        ev[1].record()
        ev[1].synchronize()
        times.append(ev[0].elapsed_time(ev[1]))
    extra = ""
    if args.op == "solve":
        u = torch.zeros_like(f)
        info = s.solve(f, u, tol=args.tol)
        levels = "".join(k for _, _, k in s.level_shapes()[1:])
        extra = " iterations=%d levels=%s min_ms=%.4f" % (info["iterations"], levels, min(times))
    print("op=%s dofs=%d precision=%s mean_ms=%.4f%s" % (args.op, n, args.precision,
                                                        sum(times) / len(times), extra))
    s.close()


def table3(args, st, inputs, torch):
    import numpy as np
    s = st.Solver(args.dim, args.degree, args.spans, args.slabs, ne_per_slab=args.ne,
                  theta=args.theta, spatial_solver="minres")
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
                its, _, _ = s.block_minres(a, c1, c2, f, u, tol=args.tol)
                steps[key] = max(steps[key], int(its[0]))
            i += 2
        else:
            i += 1
    print("table3 dim=%d spans=%s p=%d nt=%d theta=%g tol=%g max_steps_rschur=%d "
          "max_steps_complex=%d" % (args.dim, args.spans, args.degree, s.nt, args.theta, args.tol,
                                    steps["rschur"], steps["complex"]))
    s.close()


if __name__ == "__main__":
    main()
