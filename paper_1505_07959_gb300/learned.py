"""Training and evaluation of the learned coarse propagator, through the library's kernels.

    python -m paper_1505_07959_gb300.learned train --out weights/inv_wide.f32
    python -m paper_1505_07959_gb300.learned evaluate --weights weights/inv_wide.f32

Data.  Every training matrix is A = Q diag(lam) Q^T of the wide-spectrum inverse family
(lam log-uniform in [1e-2, 1], Haar Q; `inputs.sym_matrix(n, "inv_wide", seed)`).  The method
generates the trajectories: a parareal solve (fa_parareal_solve, coarse propagator the degree-4
Taylor step, i.e. the constant network c = (1, 1, 1, 1)) runs `gen_iters` iterations with the
plan's pair recorder on, so every fine sweep adds the N pairs (U^k_n, F(U^k_n)) as records
(features + 4 x 4 Gram data, computed on the GPU).  A second pass (--gen-weights) generates
records with a trained network as the coarse propagator, so that the training set also holds
the states that network's own solves visit (the late slices' states of a Taylor-4 solve are far
from them), and trains on the union (--records-in adds earlier records).

Training.  Feature standardisation (mu, sd) from the training records; network initialised with
He-scaled hidden layers, W3 = 0 and b3 = (1, 1, 1, 1) (the Taylor step); Adam on minibatches of
records, every step one fa_mlp_loss_grad and one fa_mlp_adam launch pair; the learning rate
drops tenfold for the last fifth of the steps.

Evaluation.  Solves of held-out seeds with forward-Euler G, the Taylor step and the learned G on
the same fine propagator: parareal iterations to the tolerance, device time per solve and the
relative Frobenius error of U_N against the closed-form inverse Q diag(1 / lam) Q^T.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import math
import os
import time
from typing import Dict, Sequence

import numpy as np

from . import build, fa, inputs

NF, HID, NC = fa.FA_MLP_FEATURES, fa.FA_MLP_HIDDEN, fa.FA_MLP_COEFS
REC = fa.FA_RECORD_DOUBLES
HERE = os.path.dirname(os.path.abspath(__file__))
DEFAULT_WEIGHTS = os.path.join(HERE, "weights", "inv_wide.f32")


@dataclasses.dataclass
class TrainConfig:
    ns: Sequence[int] = (256, 512, 1024)   # matrix orders, cycled over the seeds
    seeds: Sequence[int] = range(0, 64)
    kind: str = "inv_wide"
    T: float = 1.0
    N: int = 64
    J: int = 64
    dtype: str = "bf16x6"
    coarse_dtype: str = "bf16x6"           # of the generating solves (pairs are F's either way)
    gen_iters: int = 3
    steps: int = 4000
    batch: int = 1024
    lr: float = 1e-3
    seed: int = 0


def log_uniform_sizes(count: int, lo: int, hi: int, seed: int) -> list:
    """Matrix orders log-uniform in [lo, hi], rounded to integers (seeded)."""
    rng = np.random.default_rng(seed)
    return [int(round(x)) for x in np.exp(rng.uniform(math.log(lo), math.log(hi), count))]


def blob_layout() -> Dict[str, tuple]:
    """Offsets and shapes of the parameter blob (the order of the C header)."""
    shapes = [("mu", (NF,)), ("sd", (NF,)), ("W1", (HID, NF)), ("b1", (HID,)), ("W2", (HID, HID)),
              ("b2", (HID,)), ("W3", (NC, HID)), ("b3", (NC,))]
    out, off = {}, 0
    for k, s in shapes:
        out[k] = (off, s)
        off += int(np.prod(s))
    assert off == fa.FA_MLP_PARAMS
    return out


def constant_blob(c) -> np.ndarray:
    """A network whose output is c for every input (W3 = 0, b3 = c)."""
    p = np.zeros(fa.FA_MLP_PARAMS, dtype=np.float32)
    lay = blob_layout()
    p[lay["sd"][0]:lay["sd"][0] + NF] = 1.0
    o = lay["b3"][0]
    p[o:o + NC] = np.asarray(c, dtype=np.float32)
    return p


def init_blob(mu, sd, seed: int, c0=(1.0, 1.0, 1.0, 1.0)) -> np.ndarray:
    rng = np.random.default_rng(seed)
    p = constant_blob(c0)
    lay = blob_layout()

    def put(k, v):
        o, s = lay[k]
        p[o:o + int(np.prod(s))] = np.asarray(v, dtype=np.float32).ravel()
    put("mu", mu)
    put("sd", sd)
    put("W1", rng.standard_normal((HID, NF)) * math.sqrt(2.0 / NF))
    put("W2", rng.standard_normal((HID, HID)) * math.sqrt(2.0 / HID))
    return p


def generate(cfg: TrainConfig, log=None, gen_blob=None) -> np.ndarray:
    """Pair records (host float64 (R, FA_RECORD_DOUBLES)) from the method's own solves; the
    generating solves use the Taylor-4 step, or the network `gen_blob` when given (records of
    the iterates that network's own solves visit)."""
    import torch

    build.build_library()
    fa.load_library()
    out = []
    taylor = constant_blob((1.0, 1.0, 1.0, 1.0)) if gen_blob is None else np.asarray(gen_blob, dtype=np.float32)
    plans = {}
    t0 = time.time()
    for i, seed in enumerate(cfg.seeds):
        n = cfg.ns[i % len(cfg.ns)]
        if n not in plans:
            pl = fa.Plan(n, fa.FA_FLOW_INV, cfg.T, cfg.N, cfg.J, max_iters=cfg.gen_iters, tol=0.0,
                         fine_dtype=cfg.dtype,
                         coarse_dtype=cfg.dtype if cfg.dtype == "f64" else cfg.coarse_dtype,
                         coarse_kind=fa.FA_COARSE_LEARNED)
            pl.set_learned(taylor)
            pl.set_recorder(cfg.gen_iters * cfg.N)
            plans[n] = pl
        pl = plans[n]
        A = torch.from_numpy(inputs.sym_matrix(n, cfg.kind, seed).A).cuda()
        _, rep = pl.solve(A)
        out.append(pl.rec_buf[:rep["records"]].cpu().numpy())
        if log and (i + 1) % max(1, len(cfg.seeds) // 10) == 0:
            log(f"  generated {i + 1}/{len(cfg.seeds)} trajectories ({time.time() - t0:.1f} s)")
    for pl in plans.values():
        pl.close()
    return np.concatenate(out, axis=0)


def standardisation(records: np.ndarray):
    f = records[:, :NF]
    mu = f.mean(axis=0)
    sd = f.std(axis=0)
    sd = np.where(sd > 1e-9 * np.maximum(1.0, np.abs(mu)), sd, 1.0)
    return mu, sd


def train(records: np.ndarray, cfg: TrainConfig, log=None):
    """Returns (float32 blob, loss history per 10 steps)."""
    import torch

    build.build_library()
    fa.load_library()
    mu, sd = standardisation(records)
    mlp = fa.Mlp(init_blob(mu, sd, cfg.seed))
    rng = np.random.default_rng(cfg.seed + 1)
    R = records.shape[0]
    B = min(cfg.batch, R)
    per_epoch = R // B
    hist = []
    dev = None
    step = 0
    while step < cfg.steps:
        perm = rng.permutation(R)
        dev = torch.from_numpy(np.ascontiguousarray(records[perm])).cuda()
        for e in range(per_epoch):
            if step >= cfg.steps:
                break
            lr = cfg.lr if step < 0.8 * cfg.steps else 0.1 * cfg.lr
            loss, _ = mlp.loss_grad(dev[e * B:(e + 1) * B])
            mlp.adam(lr=lr)
            if step % 10 == 0:
                hist.append(float(loss.item()))
                if log and step % 500 == 0:
                    log(f"  step {step}: loss {hist[-1]:.4e}")
            step += 1
    full = torch.from_numpy(np.ascontiguousarray(records)).cuda()
    loss_all, _ = mlp.loss_grad(full)
    hist.append(float(loss_all.item()))
    return mlp.params.cpu().numpy().copy(), hist


def evaluate(params, ns=(1024,), seeds=range(1000, 1008), kind="inv_wide", T=1.0, N=64, J=64,
             tol=1e-8, dtype="bf16x6", kinds=("euler", "taylor4", "learned"), max_iters=None,
             coarse_dtype="f64", refine_steps=0, log=None) -> Dict[str, list]:
    """Per kind, per (n, seed): iterations, device ms per solve, error against A^{-1}.

    The coarse propagator runs in float64 by default: a BF16 coarse step is not smooth below
    ~2^-24 |G| and floors the convergence measure near 2e-8 on this family."""
    import torch

    build.build_library()
    fa.load_library()
    res = {k: [] for k in kinds}
    blobs = {"taylor4": constant_blob((1.0, 1.0, 1.0, 1.0)),
             "learned": None if params is None else np.asarray(params, dtype=np.float32)}
    for n in ns:
        plans = {}
        for k in kinds:
            kw = dict(max_iters=max_iters or N, tol=tol, fine_dtype=dtype,
                      coarse_dtype=dtype if dtype == "f64" else coarse_dtype,
                      refine_steps=refine_steps)
            if k == "euler":
                plans[k] = fa.Plan(n, fa.FA_FLOW_INV, T, N, J, **kw)
            else:
                plans[k] = fa.Plan(n, fa.FA_FLOW_INV, T, N, J, coarse_kind=fa.FA_COARSE_LEARNED, **kw)
                plans[k].set_learned(blobs[k])
        for seed in seeds:
            sm = inputs.sym_matrix(n, kind, seed)
            exact = (sm.Q / sm.lam[None, :]) @ sm.Q.T
            A = torch.from_numpy(sm.A).cuda()
            for k in kinds:
                X, rep = plans[k].solve(A)
                ms = rep["t_init_ms"] + rep["t_fine_ms"] + rep["t_coarse_ms"] + rep["t_refine_ms"]
                err = float(np.linalg.norm(X.cpu().numpy() - exact) / np.linalg.norm(exact))
                res[k].append({"n": n, "seed": int(seed), "iters": rep["iters"],
                               "converged": rep["converged"], "ms": ms, "err": err,
                               "g_fallback_iter": rep["g_fallback_iter"],
                               "coef_fallbacks": rep["coef_fallbacks"]})
                if log:
                    log(f"  n={n} seed={seed} {k}: {rep['iters']} iterations, {ms:.1f} ms, "
                        f"err {err:.2e}")
        for p in plans.values():
            p.close()
    return res


def summarise(res: Dict[str, list]) -> Dict[str, dict]:
    out = {}
    for k, rows in res.items():
        it = np.array([r["iters"] for r in rows], dtype=float)
        ms = np.array([r["ms"] for r in rows])
        out[k] = {"solves": len(rows), "iters_mean": float(it.mean()), "iters_max": int(it.max()),
                  "solves_per_s": float(1000.0 / ms.mean()), "ms_mean": float(ms.mean()),
                  "err_max": float(max(r["err"] for r in rows)),
                  "converged": int(sum(r["converged"] for r in rows)),
                  "fallbacks": int(sum(r["g_fallback_iter"] > 0 for r in rows))}
    return out


def main() -> None:
    ap = argparse.ArgumentParser()
    sub = ap.add_subparsers(dest="cmd", required=True)
    t = sub.add_parser("train")
    t.add_argument("--out", default=DEFAULT_WEIGHTS)
    t.add_argument("--trajectories", type=int, default=256)
    t.add_argument("--n-lo", type=int, default=256)
    t.add_argument("--n-hi", type=int, default=1024)
    t.add_argument("--N", type=int, default=64)
    t.add_argument("--J", type=int, default=64)
    t.add_argument("--gen-iters", type=int, default=3)
    t.add_argument("--steps", type=int, default=4000)
    t.add_argument("--batch", type=int, default=1024)
    t.add_argument("--lr", type=float, default=1e-3)
    t.add_argument("--dtype", default="bf16x6")
    t.add_argument("--log", default=None, help="JSON summary file")
    t.add_argument("--gen-weights", default=None, help="network blob for the generating solves")
    t.add_argument("--records-in", action="append", default=[], help=".npy records to add")
    t.add_argument("--records-out", default=None, help="save the generated records (.npy)")
    t.add_argument("--seed0", type=int, default=0, help="first training matrix seed")
    t.add_argument("--train-only", action="store_true", help="no generation: train on --records-in")
    e = sub.add_parser("evaluate")
    e.add_argument("--weights", default=DEFAULT_WEIGHTS)
    e.add_argument("--n", type=int, default=1024)
    e.add_argument("--seeds", type=int, default=8)
    e.add_argument("--seed0", type=int, default=100000)
    e.add_argument("--N", type=int, default=64)
    e.add_argument("--J", type=int, default=64)
    e.add_argument("--tol", type=float, default=1e-8)
    e.add_argument("--dtype", default="bf16x6")
    e.add_argument("--coarse-dtype", default="f64")
    e.add_argument("--refine", type=int, default=2)
    e.add_argument("--kinds", default="euler,taylor4,learned",
                   help="comma-separated coarse propagators to solve with")
    e.add_argument("--log", default=None, help="JSON summary file")
    a = ap.parse_args()
    if a.cmd == "train":
        ns = log_uniform_sizes(a.trajectories, a.n_lo, a.n_hi, 12345 + a.seed0)
        # sizes rounded to multiples of 32 keep the plans few (one per distinct order)
        ns = [max(8, int(round(x / 32)) * 32) for x in ns]
        cfg = TrainConfig(ns=ns, seeds=range(a.seed0, a.seed0 + a.trajectories), N=a.N, J=a.J,
                          dtype=a.dtype, gen_iters=a.gen_iters, steps=a.steps, batch=a.batch,
                          lr=a.lr)
        t0 = time.time()
        parts = [np.load(f) for f in a.records_in]
        if not a.train_only:
            gen_blob = None if a.gen_weights is None else np.fromfile(a.gen_weights, dtype=np.float32)
            new = generate(cfg, log=print, gen_blob=gen_blob)
            if a.records_out:
                np.save(a.records_out, new)
            parts.append(new)
        recs = np.concatenate(parts, axis=0)
        t1 = time.time()
        print(f"{recs.shape[0]} records ({a.trajectories if not a.train_only else 0} new trajectories) in {t1 - t0:.1f} s")
        params, hist = train(recs, cfg, log=print)
        t2 = time.time()
        os.makedirs(os.path.dirname(os.path.abspath(a.out)), exist_ok=True)
        params.astype(np.float32).tofile(a.out)
        summary = {"trajectories": a.trajectories, "records_in": a.records_in,
                   "gen_weights": a.gen_weights, "n_range": [a.n_lo, a.n_hi], "N": a.N,
                   "J": a.J, "dtype": a.dtype, "gen_iters": a.gen_iters, "records": int(recs.shape[0]),
                   "gen_s": t1 - t0, "train_s": t2 - t1, "steps": a.steps, "batch": a.batch,
                   "loss_first": hist[0], "loss_final_full": hist[-1]}
        print(json.dumps(summary))
        if a.log:
            with open(a.log, "w") as f:
                json.dump({"summary": summary, "loss_history": hist}, f)
    else:
        kinds = tuple(a.kinds.split(","))
        if not kinds or not set(kinds) <= {"euler", "taylor4", "learned"}:
            ap.error("--kinds takes euler, taylor4 and learned")
        params = np.fromfile(a.weights, dtype=np.float32)
        res = evaluate(params, ns=(a.n,), seeds=range(a.seed0, a.seed0 + a.seeds), N=a.N, J=a.J,
                       tol=a.tol, dtype=a.dtype, coarse_dtype=a.coarse_dtype,
                       kinds=kinds, refine_steps=a.refine, log=print)
        s = summarise(res)
        print(json.dumps(s))
        if a.log:
            with open(a.log, "w") as f:
                json.dump({"summary": s, "runs": res}, f)


if __name__ == "__main__":
    main()
