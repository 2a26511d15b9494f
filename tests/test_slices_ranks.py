"""Parareal with the slices split across ranks (paper_1505_07959_gb300.slices), on gloo ranks on
the CPU with the oracle's propagators injected: the pipelined coarse sweep and the all-reduced
stopping test must reproduce single-process Algorithm 1 iterate by iterate."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from oracle import parareal as P
from paper_1505_07959_gb300 import inputs
from paper_1505_07959_gb300 import slices


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def oracle_propagators(A, flow, T, N, m, J, count):
    """The oracle's RK4 fine propagator and Euler coarse sweep over `count` slices, on torch
    float64 CPU tensors (test-side only)."""
    dT = T / N

    def fine(U):
        return torch.stack([torch.from_numpy(P.rk4(flow, u.numpy(), A, dT, J)) for u in U])

    def coarse(V0, D, Uold):
        V, G = [V0.numpy()], []
        for i in range(count):
            g = P.euler(flow, V[i], A, dT, m)
            G.append(g)
            V.append(g if D is None else g + D[i].numpy())
        norms = None
        if Uold is not None:
            norms = torch.tensor([[np.sum((V[i + 1] - Uold[i + 1].numpy()) ** 2),
                                   np.sum(V[i + 1] ** 2)] for i in range(count)])
        return torch.from_numpy(np.stack(V)), torch.from_numpy(np.stack(G)), norms

    return fine, coarse


CASES = {"inv": (0, 1.0, 1, 4), "exp": (1, 1.0, 1, 4), "sqrt": (2, 6.0, 2, 3)}


def _rank_main(rank, ws, port, kind, N, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        flow, T, m, J = CASES[kind]
        sm = inputs.sym_matrix(7, kind, 5)
        lo, hi = slices.bounds(N, ws, rank)
        fine, coarse = oracle_propagators(sm.A, flow, T, N, m, J, hi - lo)
        comm = slices.TorchComm()
        res = slices.parareal_sliced(torch.eye(7, dtype=torch.float64), N, fine, coarse, N, 1e-12,
                                     comm)
        q.put((rank, res.lo, res.hi, res.U.numpy(), res.iterations, res.dx_history))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("ws,N,kind", [(2, 5, "inv"), (3, 7, "exp"), (2, 6, "sqrt")])
def test_sliced_parareal_equals_algorithm_1(ws, N, kind):
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, kind, N, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(ws):
        r = q.get(timeout=180)
        out[r[0]] = r[1:]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    flow, T, m, J = CASES[kind]
    sm = inputs.sym_matrix(7, kind, 5)
    ref = P.parareal(sm.A, flow, T, N, m, J, N, 1e-12)
    iters = {out[r][3] for r in range(ws)}
    assert iters == {ref.iterations}
    for r in range(ws):
        lo, hi, U, it, hist = out[r]
        assert (lo, hi) == slices.bounds(N, ws, r)
        np.testing.assert_allclose(hist, ref.dx_history, rtol=1e-10, atol=1e-300)
        for i, n in enumerate(range(lo, hi + 1)):
            assert P.rel_fro(U[i], ref.U[n]) < 1e-14, (r, n)
    # the last rank holds the result, and finite termination holds across the split
    assert P.rel_fro(out[ws - 1][2][-1], P.sequential_fine(sm.A, flow, T, N, J)) < 1e-12


def test_bounds_cover_the_slices_once():
    for N in (1, 5, 64, 127):
        for Pn in (1, 2, 3, 8):
            if Pn > N:
                continue
            spans = [slices.bounds(N, Pn, r) for r in range(Pn)]
            assert spans[0][0] == 0 and spans[-1][1] == N
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1


def _failing_rank_main(rank, ws, port, q):
    """Rank 1's fine propagator raises on the second iteration (a host-side fault); rank 0 must
    learn of it through the process group's timeout on its next collective, not hang."""
    import datetime
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws,
                            timeout=datetime.timedelta(seconds=5))
    flow, T, m, J = CASES["exp"]
    sm = inputs.sym_matrix(6, "exp", 5)
    N = 4
    lo, hi = slices.bounds(N, ws, rank)
    fine, coarse = oracle_propagators(sm.A, flow, T, N, m, J, hi - lo)
    calls = {"n": 0}

    def faulty_fine(U):
        calls["n"] += 1
        if rank == 1 and calls["n"] == 2:
            raise RuntimeError("injected fault in the fine propagator")
        return fine(U)

    try:
        slices.parareal_sliced(torch.eye(6, dtype=torch.float64), N, faulty_fine, coarse, N, 0.0,
                               slices.TorchComm())
        q.put((rank, "finished"))
    except RuntimeError as e:
        q.put((rank, "injected" if "injected" in str(e) else "peer-error"))
    except Exception:
        q.put((rank, "peer-error"))


def test_a_failing_rank_is_detected_by_its_peers():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_failing_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    out = dict(q.get(timeout=120) for _ in range(ws))
    for p in procs:
        p.join(60)
    assert out[1] == "injected"
    assert out[0] == "peer-error"           # the all-reduce (or receive) timed out with an error
