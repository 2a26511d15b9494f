"""Classical parareal with the time slices split across ranks (one process per GPU).

Algorithm 1 of the paper (Section 2) evaluates the fine propagator on every slice in parallel
and then runs the cheap coarse propagator as a sequential sweep.  Split over P ranks, rank r
owns the slices n in [lo_r, hi_r), lo_r = r N / P, and the states U_lo .. U_hi at their ends:

  Step 0 (eq. eqStep0)   rank r receives U^0_lo from rank r - 1 (rank 0 starts from X0), runs
                         G over its slices, U^0_{n+1} = G(U^0_n), and sends U^0_hi to rank r + 1;
  Step k+1               every rank computes F(U^k_n) on its own slices at once (no exchange),
                         then the correction sweep U^{k+1}_{n+1} = G(U^{k+1}_n) + D_n with
                         D_n = F(U^k_n) - G(U^k_n) (eq. eqStepk+1) passes along the ranks as a
                         pipeline: receive U^{k+1}_lo, sweep, send U^{k+1}_hi;
  stopping test          max over n = 1..N of ||U^{k+1}_n - U^k_n||_F / ||U^{k+1}_n||_F: each
                         rank forms the maximum over its own n in (lo, hi], and one all-reduce
                         (max) of that scalar gives every rank the same decision.

So each iteration moves one n x n matrix across each rank boundary and one scalar through an
all-reduce; the fine sweep, which holds all of the flops, needs no communication.  The last
rank's U_N is the result.

The propagators are injected: `fine(U_starts) -> F` maps the rank's slice starts (its own
[count][n][n] tensor) to their fine images, and `coarse(V_lo, D) -> (V, G, norms)` runs the
rank's coarse sweep from V_lo with corrections D (None for Step 0), returning V_lo .. V_hi,
G(V_n) for the rank's slices and, when `Uold` is given, per slice ||V_{n+1} - Uold_{n+1}||^2 and
||V_{n+1}||^2.  `LibraryPropagators` provides both from a libfa plan built for the rank's slice
count (the flows are autonomous, so a plan over N_r slices of the same length dT is the rank's
share of the whole problem); tests inject the CPU oracle's propagators instead.  Communication
goes through torch.distributed (gloo for CPU tensors, NCCL for device tensors) or any object
with the same four methods (`rank`, `size`, `send`, `recv`, `max`).
"""
from __future__ import annotations

import dataclasses
from typing import Callable, List, Optional, Tuple

import torch


def bounds(N: int, P: int, r: int) -> Tuple[int, int]:
    """Slices [lo, hi) of rank r when N slices are split over P ranks (sizes differ by <= 1)."""
    return r * N // P, (r + 1) * N // P


class TorchComm:
    """Point-to-point and max-reduction through an initialised torch.distributed group."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group)
        self.size = dist.get_world_size(group)

    def send(self, t: torch.Tensor, dst: int) -> None:
        self.dist.send(t.contiguous(), dst, group=self.group)

    def recv(self, t: torch.Tensor, src: int) -> None:
        self.dist.recv(t, src, group=self.group)

    def max(self, x: float, device) -> float:
        v = torch.tensor([x], dtype=torch.float64, device=device)
        self.dist.all_reduce(v, op=self.dist.ReduceOp.MAX, group=self.group)
        return float(v.item())


@dataclasses.dataclass
class SlicedResult:
    lo: int
    hi: int
    U: torch.Tensor                   # this rank's U_lo .. U_hi of the last iterate
    iterations: int
    dx_history: List[float]           # the global stopping measure of every iteration

    def final(self, N: int) -> Optional[torch.Tensor]:
        """U_N on the rank that owns the last slice, else None."""
        return self.U[-1] if self.hi == N else None


def parareal_sliced(X0: torch.Tensor, N: int, fine: Callable, coarse: Callable, K_max: int,
                    tol: float, comm) -> SlicedResult:
    """Algorithm 1 over this rank's slices (module docstring).  X0 is needed on rank 0 only
    (other ranks may pass any tensor of the state's shape, dtype and device)."""
    r, P = comm.rank, comm.size
    lo, hi = bounds(N, P, r)
    if hi <= lo:
        raise ValueError(f"rank {r} has no slice (N = {N} < {P} ranks)")
    shape, dev = tuple(X0.shape), X0.device

    def start_state() -> torch.Tensor:
        if r == 0:
            return X0.clone()
        v = torch.empty(shape, dtype=X0.dtype, device=dev)
        comm.recv(v, r - 1)
        return v

    def pass_on(V: torch.Tensor) -> None:
        if r + 1 < P:
            comm.send(V[-1], r + 1)

    # Step 0 (eq. eqStep0): U^0_{n+1} = G(U^0_n), G(U^0_n) kept for the first correction
    U, Gold, _ = coarse(start_state(), None, None)
    pass_on(U)
    hist: List[float] = []
    it = 0
    for _ in range(K_max):
        # Step k+1: the fine propagator on this rank's slices at once ...
        D = fine(U[:-1]) - Gold
        # ... then the correction sweep, pipelined along the ranks (eq. eqStepk+1)
        V, Gnew, norms = coarse(start_state(), D, U)
        pass_on(V)
        local = torch.sqrt(norms[:, 0] / norms[:, 1]).max().item()
        if local != local:                       # NaN: make the maximum non-finite everywhere
            local = float("inf")
        dx = comm.max(local, norms.device)
        U, Gold = V, Gnew
        it += 1
        hist.append(dx)
        if dx < tol:
            break
    return SlicedResult(lo=lo, hi=hi, U=U, iterations=it, dx_history=hist)


class LibraryPropagators:
    """The rank's fine and coarse sweeps through libfa: a plan over the rank's N_r slices with
    horizon N_r dT (the flows are autonomous, so each slice is the same map whatever its
    index)."""

    def __init__(self, plan):
        self.plan = plan

    def fine(self, U: torch.Tensor) -> torch.Tensor:
        return self.plan.fine_sweep(U)

    def coarse(self, V0: torch.Tensor, D: Optional[torch.Tensor], Uold: Optional[torch.Tensor]):
        return self.plan.coarse_sweep(V0, D, Uold)


def library_plan(n: int, flow: int, T: float, N: int, rank: int, size: int, **kw):
    """A libfa plan (fa.Plan) for rank `rank`'s share of an N-slice problem on [0, T]."""
    from . import fa
    lo, hi = bounds(N, size, rank)
    return fa.Plan(n, flow, T * (hi - lo) / N, hi - lo, **kw)
