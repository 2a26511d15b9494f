"""The bench's multi-rank host logic on two gloo ranks (CPU): barrier, the max-over-ranks job
rate, per-rank independent problems, and the reference arm printing on rank 0 only."""
import io
import os
import socket
import contextlib

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(ws), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    try:
        assert bench._dist() == (ws, rank, rank)
        bench._barrier(ws)
        rate, t = bench._job_rate(3, 1.0 + rank, ws, torch.device("cpu"))
        seed = bench._rank_seed(rank)
        buf = io.StringIO()
        with contextlib.redirect_stdout(buf):
            class A:
                gpus, steps, warmup = ws, 1, 0
            if rank != 0:
                bench.run_reference(A)          # ranks other than 0 return without work
        q.put((rank, rate, t, seed, buf.getvalue()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    ws, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    out = dict((r[0], r[1:]) for r in (q.get(timeout=10) for _ in range(ws)))
    for r in range(ws):
        rate, t, seed, printed = out[r]
        assert t == 2.0 and rate == pytest.approx(ws * 3 / 2.0)   # slowest rank's time
        assert printed == ""
    assert out[0][2] != out[1][2]                                  # independent problems


def test_bench_float64_iteration_count_is_the_oracles():
    """The float64 GPU baseline in the bench line extrapolates with the float64 parareal's
    iteration count to the workload's tolerance (1e-10); the eigenvalue-space oracle fixes it."""
    import bench
    from oracle import scalar as S
    from paper_1505_07959_gb300 import inputs
    w = bench.WORK
    sm = inputs.sym_matrix(w.n, w.kind, w.seed)
    r = S.parareal(sm.lam, w.flow, w.T, w.N, w.m, w.J, w.K_max, w.tol)
    assert r.iterations == bench.FP64_ITERS
