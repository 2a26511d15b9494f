"""Run fine sweeps of one shape on the GPU (for profiling and quick timing).

    python -m paper_1505_07959_gb300.sweep_case --flow exp --n 2048 --N 16 --J 1 --dtype bf16x6

Builds the library if needed, loads A = Q diag(lam) Q^T of the flow's family (seed 0), runs
`--sweeps` fine sweeps from U_b = I for every slice b, and prints the per-launch time of the
tensor-core GEMM (one launch per RK4 stage; two per stage for the inverse flow).
"""
from __future__ import annotations

import argparse

from . import build, fa, inputs

FLOWS = {"inv": (fa.FA_FLOW_INV, "inv"), "exp": (fa.FA_FLOW_EXP, "exp"),
         "sqrt": (fa.FA_FLOW_SQRT, "sqrt")}


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--flow", default="exp", choices=sorted(FLOWS))
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--N", type=int, default=16)
    ap.add_argument("--J", type=int, default=1)
    ap.add_argument("--T", type=float, default=1.0)
    ap.add_argument("--dtype", default="bf16x6")
    ap.add_argument("--sweeps", type=int, default=2)
    args = ap.parse_args()

    import torch

    build.build_library()
    fa.load_library()
    flow, kind = FLOWS[args.flow]
    sm = inputs.sym_matrix(args.n, kind, 0)
    plan = fa.Plan(args.n, flow, args.T, args.N, fine_steps=args.J, fine_dtype=args.dtype)
    plan.set_matrix(torch.from_numpy(sm.A).cuda())
    U = torch.eye(args.n, dtype=torch.float64, device="cuda").expand(args.N, args.n, args.n).contiguous()
    F = torch.empty_like(U)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.sweeps):
        fa.fa_fine_sweep(plan.handle, U, F)
    e1.record()
    torch.cuda.synchronize()
    launches = args.sweeps * 4 * args.J * (2 if args.flow == "inv" else 1)
    print(f"{args.flow} n={args.n} N={args.N} J={args.J} {args.dtype}: "
          f"{e0.elapsed_time(e1) / launches:.3f} ms per GEMM launch ({launches} launches)")
    plan.close()


if __name__ == "__main__":
    main()
