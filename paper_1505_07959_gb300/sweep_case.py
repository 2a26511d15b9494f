"""Run fine sweeps of one shape on the GPU (for profiling and quick timing).

    python -m paper_1505_07959_gb300.sweep_case --flow exp --n 2048 --N 16 --J 1 --dtype bf16x6
    python -m paper_1505_07959_gb300.sweep_case --flow sqrt --n 4096 --N 8 --T 20 --dtype bf16 --counters
    python -m paper_1505_07959_gb300.sweep_case --flow exp --n 2048 --N 64 --coarse --counters

Builds the library if needed, loads A = Q diag(lam) Q^T of the flow's family (seed 0), runs
`--sweeps` fine sweeps from U_b = I for every slice b, and prints the per-launch time of the
tensor-core GEMM (one launch per RK4 stage; two per stage for the inverse flow).  With --coarse
it times correction sweeps instead (one single-slice launch per slice and Euler step).  With
--counters, one more sweep runs with the kernel's per-role cycle counters on
(fa_debug_set_profile) and prints them per tile, in thousands of cycles, summed over the CTAs
and divided by the tiles: the waits of each role, the drain's and the epilogue's busy time, and
the kernel's cycles.
"""
from __future__ import annotations

import argparse
import json

from . import build, fa, inputs

FLOWS = {"inv": (fa.FA_FLOW_INV, "inv"), "exp": (fa.FA_FLOW_EXP, "exp"),
         "sqrt": (fa.FA_FLOW_SQRT, "sqrt")}
# the counter words of fa_debug_set_profile, in order
COUNTERS = ["producer_wait_slots", "mma_wait_tiles", "mma_wait_main_chunk", "mma_wait_corr",
            "drain_wait_main_chunk", "drain_wait_corr", "drain_wait_fin_buffer",
            "epilogue_wait_tile", "epilogue_busy", "drain_busy", "kernel"]


def main() -> None:
    ap = argparse.ArgumentParser()
    ap.add_argument("--flow", default="exp", choices=sorted(FLOWS))
    ap.add_argument("--n", type=int, default=2048)
    ap.add_argument("--N", type=int, default=16)
    ap.add_argument("--J", type=int, default=1)
    ap.add_argument("--T", type=float, default=1.0)
    ap.add_argument("--dtype", default="bf16x6")
    ap.add_argument("--sweeps", type=int, default=2)
    ap.add_argument("--coarse-dtype", default=None, help="needed with --dtype fp8e4m3 (bf16)")
    ap.add_argument("--counters", action="store_true", help="print the per-role cycle counters")
    ap.add_argument("--coarse", action="store_true",
                    help="time coarse sweeps (correction and norms, one launch per slice) instead")
    args = ap.parse_args()

    import torch

    build.build_library()
    fa.load_library()
    flow, kind = FLOWS[args.flow]
    sm = inputs.sym_matrix(args.n, kind, 0)
    plan = fa.Plan(args.n, flow, args.T, args.N, fine_steps=args.J, fine_dtype=args.dtype,
                   coarse_dtype=args.coarse_dtype)
    plan.set_matrix(torch.from_numpy(sm.A).cuda())
    U = torch.eye(args.n, dtype=torch.float64, device="cuda").expand(args.N, args.n, args.n).contiguous()
    F = torch.empty_like(U)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if args.coarse:
        # the correction sweep of an iteration: V_{n+1} = G(V_n) + D_n with norms against U
        D = torch.zeros_like(U)
        Uo = torch.eye(args.n, dtype=torch.float64, device="cuda").expand(args.N + 1, args.n,
                                                                          args.n).contiguous()
        Un = torch.empty_like(Uo)
        Gn = torch.empty_like(U)
        nrm = torch.empty((args.N, 2), dtype=torch.float64, device="cuda")

        def sweep():
            fa.fa_coarse_sweep(plan.handle, Uo[0], D, Un, Gn, nrm, Uo)
    else:
        def sweep():
            fa.fa_fine_sweep(plan.handle, U, F)
    sweep()
    torch.cuda.synchronize()
    e0.record()
    for _ in range(args.sweeps):
        sweep()
    e1.record()
    torch.cuda.synchronize()
    if args.coarse:
        launches = args.sweeps * args.N * (2 if args.flow == "inv" else 1)
    else:
        launches = args.sweeps * 4 * args.J * (2 if args.flow == "inv" else 1)
    print(f"{args.flow} n={args.n} N={args.N} J={args.J} {args.dtype}: "
          f"{e0.elapsed_time(e1) / launches:.3f} ms per GEMM launch ({launches} launches)")
    if args.counters:
        cnt = torch.zeros(16, dtype=torch.int64, device="cuda")
        fa.fa_debug_set_profile(cnt)
        sweep()
        torch.cuda.synchronize()
        fa.fa_debug_set_profile(None)
        c = cnt.cpu().tolist()
        tiles = max(c[11], 1)
        print(json.dumps({name: round(c[k] / tiles / 1e3, 2) for k, name in enumerate(COUNTERS)}
                         | {"tiles": c[11]}))
    plan.close()


if __name__ == "__main__":
    main()
