"""Learned coarse propagator on the GPU against its float64 oracle.

Records (features and Gram data), the network's forward pass, loss and gradient (the gradient
check of the training kernels), Adam, the learned coarse sweep, whole solves with the learned G,
both fallbacks to forward Euler, the in-solve recorder, and a small end-to-end training run that
must beat Euler G.
"""
import math

import numpy as np
import pytest

from oracle import learned as L, parareal as P
from paper_1505_07959_gb300 import fa, inputs
from tests.gpu_helpers import cuda_or_fail, dev, host

pytestmark = pytest.mark.gpu

KIND = {fa.FA_FLOW_INV: "inv_wide", fa.FA_FLOW_EXP: "exp"}


def _random_params(seed, w3_scale=0.05):
    """A network with non-trivial output (random W3), features standardised near unit scale."""
    p = L.init_params(seed)
    rng = np.random.default_rng(seed + 100)
    p["W3"] = rng.standard_normal(p["W3"].shape) * w3_scale
    p["b3"] = np.array([1.0, 1.0, 1.0, 1.0])
    p["mu"] = np.array([0.5, 0.06, 0.0, 1.0, 0.2, 2.0, 1.5, 2.0])
    p["sd"] = np.array([0.3, 0.05, 0.5, 0.5, 0.1, 2.0, 2.0, 2.0])
    return p


def _sensible_params(flow, A, T, N, seed, w3=0.01):
    """A network standardised on the features of the Taylor-step trajectory of A, with a small
    random last layer: coefficients within a few percent of (1, 1, 1, 1)."""
    p = L.init_params(seed)
    Z = L.probes(A.shape[0])
    X = np.eye(A.shape[0])
    feats = []
    for s in range(N):
        feats.append(L.features(flow, A, X, s / N, T / N, Z))
        X = L.g_theta(flow, A, X, T / N, [1, 1, 1, 1])
    f = np.array(feats)
    sd = f.std(axis=0)
    p["mu"], p["sd"] = f.mean(axis=0), np.where(sd > 1e-9, sd, 1.0)
    p["W3"] = np.random.default_rng(seed + 7).standard_normal(p["W3"].shape) * w3
    p["b3"] = np.ones(4)
    return L.from_blob(L.to_blob(p))


def _const_params(c):
    p = L.init_params(0)
    p["b3"] = np.asarray(c, dtype=float)
    return p


def _oracle_records(flow, A, U, F, dT):
    Z = L.probes(A.shape[0])
    g, ta = L.gershgorin(A), L.hutchinson(A, Z)
    N = len(U)
    out = np.zeros((N, fa.FA_RECORD_DOUBLES))
    for b in range(N):
        out[b, :8] = L.features(flow, A, U[b], b / N, dT, Z, g, ta)
        M, v, dd = L.pair_record(flow, A, U[b], F[b], dT)
        out[b, 8:24] = M.ravel()
        out[b, 24:28] = v
        out[b, 28] = dd
    return out


def _states(flow, A, T, N, J):
    """Oracle states U_b (the Euler Step-0 trajectory) and their fine images F(U_b)."""
    dT = T / N
    U = [np.eye(A.shape[0])]
    for _ in range(N - 1):
        U.append(P.euler(flow, U[-1], A, dT, 1))
    F = [P.rk4(flow, u, A, dT, J) for u in U]
    return np.array(U), np.array(F)


def _check_records(got, want, mixed):
    for b in range(got.shape[0]):
        g, w = got[b], want[b]
        # features: exact up to rounding, except ||Fl(X)|| (a product) in mixed arithmetic
        ftol = np.full(8, 1e-12)
        if mixed:
            ftol[6] = 1e-5
        assert np.all(np.abs(g[:8] - w[:8]) <= ftol * np.maximum(1.0, np.abs(w[:8]))), (b, g[:8], w[:8])
        M, Mw = g[8:24].reshape(4, 4), w[8:24].reshape(4, 4)
        d = np.sqrt(np.diag(Mw))
        tol = 2e-5 if mixed else 1e-11
        assert np.all(np.abs(M - Mw) <= tol * np.outer(d, d)), (b, M, Mw)
        dd = w[28]
        assert np.all(np.abs(g[24:28] - w[24:28]) <= tol * d * math.sqrt(dd)), (b, g[24:28], w[24:28])
        assert abs(g[28] - dd) <= 1e-12 * dd
        assert np.all(g[29:] == 0)


@pytest.mark.parametrize("flow", [fa.FA_FLOW_INV, fa.FA_FLOW_EXP])
@pytest.mark.parametrize("dtype,n", [("f64", 72), ("bf16x6", 136)])
def test_records_match_oracle(flow, dtype, n):
    cuda_or_fail()
    sm = inputs.sym_matrix(n, KIND[flow], 21 + n)
    T, N, J = 1.0, 4, 4
    U, F = _states(flow, sm.A, T, N, J)
    plan = fa.Plan(n, flow, T, N, J, fine_dtype=dtype)
    plan.set_matrix(dev(sm.A))
    got = host(plan.records(dev(U), dev(F)))
    _check_records(got, _oracle_records(flow, sm.A, U, F, T / N), dtype != "f64")
    plan.close()


def test_records_of_degenerate_pairs():
    """D = 0 (F equal to U) gives dd = 0 and v = 0; the features still follow U."""
    cuda_or_fail()
    n, N = 40, 2
    sm = inputs.sym_matrix(n, "inv_wide", 5)
    U = np.array([np.eye(n), 2 * np.eye(n)])
    plan = fa.Plan(n, 0, 1.0, N, 2)
    plan.set_matrix(dev(sm.A))
    got = host(plan.records(dev(U), dev(U)))
    assert np.all(got[:, 24:29] == 0.0)
    Z = L.probes(n)
    assert abs(got[1, 5] - L.hutchinson(U[1], Z) / n) < 1e-14
    plan.close()


def test_mlp_forward_matches_oracle():
    cuda_or_fail()
    p = _random_params(3)
    rng = np.random.default_rng(4)
    B = 37                                             # ragged against 8-sample blocks
    feat = p["mu"] + p["sd"] * rng.standard_normal((B, 8))
    mlp = fa.Mlp(L.to_blob(p))
    got = host(mlp.forward(dev(feat)))
    want, _ = L.forward(L.deployed(L.from_blob(L.to_blob(p))), feat)
    assert np.max(np.abs(got - want)) <= 1e-5 * np.max(np.abs(want))
    # the records' layout: features are the first 8 doubles of each row
    rec = np.zeros((B, fa.FA_RECORD_DOUBLES))
    rec[:, :8] = feat
    assert np.array_equal(host(mlp.forward(dev(rec))), got)


def _random_records(B, seed):
    rng = np.random.default_rng(seed)
    rec = np.zeros((B, fa.FA_RECORD_DOUBLES))
    p = _random_params(0)
    rec[:, :8] = p["mu"] + p["sd"] * rng.standard_normal((B, 8))
    for b in range(B):
        Z = rng.standard_normal((4, 30)) * np.array([1.0, 0.3, 0.1, 0.03])[:, None]
        D = Z.T @ np.array([1.0, 1.1, 0.9, 1.3]) + 0.05 * rng.standard_normal(30)
        rec[b, 8:24] = (Z @ Z.T).ravel()
        rec[b, 24:28] = Z @ D
        rec[b, 28] = D @ D
    return rec


def test_mlp_gradient_check_against_oracle():
    """The training kernels' loss and gradient against the float64 oracle at the BF16 weight
    values (the oracle's backprop is itself pinned by finite differences)."""
    cuda_or_fail()
    B = 301
    rec = _random_records(B, 7)
    p = L.from_blob(L.to_blob(_random_params(5, w3_scale=0.2)))
    mlp = fa.Mlp(L.to_blob(p))
    loss, grad = mlp.loss_grad(dev(rec))
    loss, grad = float(host(loss)[0]), host(grad).astype(np.float64)
    M, v, dd = rec[:, 8:24].reshape(B, 4, 4), rec[:, 24:28], rec[:, 28]
    want_loss, g = L.loss_and_grad(L.deployed(p), rec[:, :8], M, v, dd)
    assert abs(loss - want_loss) <= 1e-5 * abs(want_loss)
    gd = L.from_blob(grad)
    assert np.all(gd["mu"] == 0) and np.all(gd["sd"] == 0)
    for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
        err = np.max(np.abs(gd[k] - g[k]))
        assert err <= 1e-4 * np.max(np.abs(g[k])) + 1e-12, (k, err, np.max(np.abs(g[k])))
    # bitwise reproducible
    _, grad2 = mlp.loss_grad(dev(rec))
    assert np.array_equal(host(grad2), grad.astype(np.float32))


def test_adam_matches_oracle():
    cuda_or_fail()
    B = 64
    rec = _random_records(B, 9)
    p0 = L.from_blob(L.to_blob(_random_params(6, w3_scale=0.2)))
    mlp = fa.Mlp(L.to_blob(p0))
    q = {k: v.copy() for k, v in p0.items()}
    st = {}
    for _ in range(3):
        _, grad = mlp.loss_grad(dev(rec))
        g = L.from_blob(host(grad))
        mlp.adam(lr=1e-3)
        q = L.adam(q, g, st, lr=1e-3)
        got = L.from_blob(host(mlp.params))
        for k in ("W1", "b1", "W2", "b2", "W3", "b3"):
            assert np.max(np.abs(got[k] - q[k])) <= 2e-6 * max(1.0, np.max(np.abs(q[k])))
        q = {k: got[k].copy() for k in got}       # continue from the GPU's float32 values
    assert np.array_equal(got["mu"], p0["mu"]) and np.array_equal(got["sd"], p0["sd"])


def _learned_plan(n, flow, T, N, J, params, dtype="f64", **kw):
    plan = fa.Plan(n, flow, T, N, J, fine_dtype=dtype, coarse_kind=fa.FA_COARSE_LEARNED, **kw)
    plan.set_learned(L.to_blob(params))
    return plan


@pytest.mark.parametrize("flow", [fa.FA_FLOW_INV, fa.FA_FLOW_EXP])
def test_constant_network_coarse_sweep_f64(flow):
    """W3 = 0: c = b3 exactly, and the sweep is the oracle's G_theta chain with correction."""
    cuda_or_fail()
    n, T, N = 70, 1.0, 5
    sm = inputs.sym_matrix(n, KIND[flow], 31)
    c = np.float32([0.9, 1.2, 0.7, 1.5]).astype(np.float64)    # the blob holds float32
    plan = _learned_plan(n, flow, T, N, 2, _const_params(c))
    plan.set_matrix(dev(sm.A))
    U, G, _ = plan.coarse_sweep(dev(np.eye(n)))
    dT = T / N
    Uo = [np.eye(n)]
    for s in range(N):
        Uo.append(L.g_theta(flow, sm.A, Uo[-1], dT, c))
    for s in range(N):
        assert P.rel_fro(host(U[s + 1]), Uo[s + 1]) < 1e-12
        assert P.rel_fro(host(G[s]), Uo[s + 1]) < 1e-12
    assert np.array_equal(host(plan.learned_coefs()), np.tile(np.float32(c), (N, 1)))
    # with a correction and norms
    rng = np.random.default_rng(2)
    D = 1e-3 * rng.standard_normal((N, n, n))
    Uold = host(U)
    U2, G2, norms = plan.coarse_sweep(dev(np.eye(n)), D=dev(D), Uold=dev(Uold))
    V = [np.eye(n)]
    for s in range(N):
        g = L.g_theta(flow, sm.A, V[-1], dT, c)
        assert P.rel_fro(host(G2[s]), g) < 1e-12
        V.append(g + D[s])
    nh = host(norms)
    for s in range(N):
        assert P.rel_fro(host(U2[s + 1]), V[s + 1]) < 1e-12
        assert abs(nh[s, 0] - np.sum((V[s + 1] - Uold[s + 1]) ** 2)) <= 1e-10 * nh[s, 0]
        assert abs(nh[s, 1] - np.sum(V[s + 1] ** 2)) <= 1e-12 * nh[s, 1]
    plan.close()


def test_network_coarse_sweep_follows_oracle_coefficients():
    cuda_or_fail()
    n, T, N = 96, 1.0, 6
    sm = inputs.sym_matrix(n, "inv_wide", 41)
    p = L.from_blob(L.to_blob(_random_params(8)))
    plan = _learned_plan(n, fa.FA_FLOW_INV, T, N, 2, p)
    plan.set_matrix(dev(sm.A))
    U, _, _ = plan.coarse_sweep(dev(np.eye(n)))
    coefs = host(plan.learned_coefs())
    G = L.learned_G(p, 0, sm.A, T, N)
    Z = L.probes(n)
    X = np.eye(n)
    for s in range(N):
        Xg = host(U[s])
        # float32 coefficients move G by ~1e-7 * dT * |Fl(X)| per slice
        assert P.rel_fro(Xg, X) < 1e-6
        c_or = L.coefficients(p, L.features(0, sm.A, Xg, s / N, T / N, Z))
        assert np.max(np.abs(coefs[s] - c_or)) <= 1e-5 * np.max(np.abs(c_or)), (s, coefs[s], c_or)
        assert np.max(np.abs(coefs[s] - 1.0)) > 1e-3       # the network is not constant
        X = G(s, X)
    plan.close()


@pytest.mark.parametrize("flow", [fa.FA_FLOW_INV, fa.FA_FLOW_EXP])
def test_learned_solve_f64_matches_oracle(flow):
    cuda_or_fail()
    n, T, N, J = 64, 1.0, 8, 8
    sm = inputs.sym_matrix(n, KIND[flow], 51)
    p = _sensible_params(flow, sm.A, T, N, 9)
    plan = _learned_plan(n, flow, T, N, J, p, max_iters=N, tol=1e-10)
    X, rep = plan.solve(dev(sm.A))
    ro = L.parareal_learned(p, sm.A, flow, T, N, J, N, 1e-10)
    assert rep["status"] == fa.FA_OK and rep["converged"]
    assert abs(rep["iters"] - ro.iterations) <= 1
    assert P.rel_fro(host(X), ro.U[N]) < 1e-9
    # the converged result does not depend on G
    pe = fa.Plan(n, flow, T, N, J, max_iters=N, tol=1e-10)
    Xe, _ = pe.solve(dev(sm.A))
    assert P.rel_fro(host(X), host(Xe)) < 1e-8
    assert rep["coef_fallbacks"] == 0 and rep["g_fallback_iter"] == 0
    plan.close()
    pe.close()


def test_nonfinite_coefficients_fall_back_to_euler():
    cuda_or_fail()
    n, T, N, J = 48, 1.0, 6, 6
    sm = inputs.sym_matrix(n, "inv_wide", 61)
    plan = _learned_plan(n, 0, T, N, J, _const_params([np.nan, 1.0, 1.0, 1.0]), max_iters=N,
                         tol=1e-10)
    X, rep = plan.solve(dev(sm.A))
    pe = fa.Plan(n, 0, T, N, J, max_iters=N, tol=1e-10)
    Xe, repe = pe.solve(dev(sm.A))
    assert rep["iters"] == repe["iters"]
    # every learned coarse step fell back: Step 0 and each iteration until (if ever) the
    # growing-dx rule switched the solve to Euler G
    learned_sweeps = 1 + (rep["g_fallback_iter"] or rep["iters"])
    assert rep["coef_fallbacks"] == N * learned_sweeps
    assert P.rel_fro(host(X), host(Xe)) < 1e-13
    assert np.all(host(plan.learned_coefs()) == np.float32([1, 0, 0, 0]))
    plan.close()
    pe.close()


def test_growing_dx_switches_to_euler_and_still_terminates():
    """c = (3, 0, 0, 0) on the exponential flow makes dx grow at iteration 2; the rest runs with
    Euler G and, by finite termination, N iterations give the sequential fine solution."""
    cuda_or_fail()
    n, T, N, J = 64, 1.0, 8, 8
    sm = inputs.sym_matrix(n, "exp", 3)
    plan = _learned_plan(n, 1, T, N, J, _const_params([3.0, 0.0, 0.0, 0.0]), max_iters=N, tol=0.0)
    X, rep = plan.solve(dev(sm.A))
    assert rep["g_fallback_iter"] == 2
    assert rep["dx_history"][1] > rep["dx_history"][0]
    assert P.rel_fro(host(X), P.sequential_fine(sm.A, 1, T, N, J)) < 1e-12
    plan.close()


def test_first_iteration_guard_switches_to_euler_when_worse():
    """The opt-in guard: with c = (0.5, 0, 0, 0) on the exponential flow the first convergence
    measure (0.75 in the oracle) exceeds Euler G's (0.09), so the solve continues with Euler G
    from iteration 1 and, by finite termination, N iterations give the sequential fine solution;
    without the guard nothing falls back.  With the Taylor-4 step (first measure 1.3e-4) the
    guard does not fire and leaves the solve bitwise unchanged."""
    cuda_or_fail()
    n, T, N, J = 64, 1.0, 8, 8
    sm = inputs.sym_matrix(n, "exp", 3)
    pe = fa.Plan(n, 1, T, N, J, max_iters=N, tol=0.0)
    _, repe = pe.solve(dev(sm.A))
    pe.close()
    seq = P.sequential_fine(sm.A, 1, T, N, J)
    for c, fires in (([0.5, 0.0, 0.0, 0.0], True), ([1.0, 1.0, 1.0, 1.0], False)):
        plan = _learned_plan(n, 1, T, N, J, _const_params(c), max_iters=N, tol=0.0)
        X0, rep0 = plan.solve(dev(sm.A))
        plan.set_learned_check(True)
        X, rep = plan.solve(dev(sm.A))
        assert rep0["g_fallback_iter"] != 1
        if fires:
            assert rep["g_fallback_iter"] == 1, rep
            assert rep["dx_history"][0] > repe["dx_history"][0]
            assert P.rel_fro(host(X), seq) < 1e-12
        else:
            # (the growing-dx rule may still act at rounding level, the same way in both solves)
            assert rep["g_fallback_iter"] == rep0["g_fallback_iter"] != 1
            assert rep["dx_history"][0] < repe["dx_history"][0]
            assert np.array_equal(host(X), host(X0))
        plan.close()
    euler_plan = fa.Plan(n, 1, T, N, J, max_iters=N, tol=0.0)
    with pytest.raises(fa.FaError) as e:
        euler_plan.set_learned_check(True)
    assert e.value.status == 1
    euler_plan.close()


def test_recorder_collects_the_solve_pairs():
    cuda_or_fail()
    n, T, N, J = 56, 1.0, 4, 4
    sm = inputs.sym_matrix(n, "inv_wide", 71)
    plan = fa.Plan(n, 0, T, N, J, max_iters=3, tol=0.0)
    buf = plan.set_recorder(4 * N)
    X, rep = plan.solve(dev(sm.A))
    assert rep["iters"] == 3 and rep["records"] == 3 * N
    got = host(buf)
    assert np.all(got[3 * N:] == 0)
    # iteration 1's pairs are (U^0_n, F(U^0_n)) with U^0 the Euler Step-0 trajectory
    U, F = _states(0, sm.A, T, N, J)
    _check_records(got[:N], _oracle_records(0, sm.A, U, F, T / N), False)
    plan.close()


def test_training_beats_euler_on_held_out_matrices():
    """End to end: pairs from the method's own solves, training by the GPU kernels, and fewer
    parareal iterations than Euler G on held-out matrices of the same family."""
    cuda_or_fail()
    from paper_1505_07959_gb300 import learned as LG
    cfg = LG.TrainConfig(ns=(48, 64, 80), seeds=range(100, 112), N=16, J=16, dtype="f64",
                         gen_iters=4, steps=600, batch=256, lr=2e-3)
    recs = LG.generate(cfg)
    assert recs.shape[0] == len(cfg.seeds) * cfg.gen_iters * cfg.N
    params, hist = LG.train(recs, cfg)
    assert hist[-1] < 0.5 * hist[0]
    res = LG.evaluate(params, ns=(64,), seeds=range(900, 903), N=16, J=16, tol=1e-8,
                      dtype="f64", kinds=("euler", "taylor4", "learned"))
    it = {k: np.mean([r["iters"] for r in res[k]]) for k in res}
    assert it["learned"] < it["euler"], it
    assert it["learned"] <= it["taylor4"], it
    for re_, rl in zip(res["euler"], res["learned"]):
        # the same fine solution (RK4 error ~1e-4 at this resolution) to the tolerance
        assert abs(rl["err"] - re_["err"]) < 1e-7 and rl["converged"]


@pytest.mark.parametrize("flow,n", [(fa.FA_FLOW_INV, 136), (fa.FA_FLOW_EXP, 200)])
def test_mixed_constant_network_coarse_sweep(flow, n):
    """BF16x6 Taylor-term chain (EPI_TAYLOR epilogues) against the float64 G_theta chain."""
    cuda_or_fail()
    T, N = 1.0, 4
    # the narrow inverse family keeps dT |BX| < 1: the Taylor terms shrink and the check reads
    # the products' accuracy, not the amplification of a divergent series
    sm = inputs.sym_matrix(n, "inv" if flow == fa.FA_FLOW_INV else "exp", 33)
    c = np.float32([1.0, 1.1, 0.8, 1.3]).astype(np.float64)
    plan = _learned_plan(n, flow, T, N, 2, _const_params(c), dtype="bf16x6")
    plan.set_matrix(dev(sm.A))
    U, G, _ = plan.coarse_sweep(dev(np.eye(n)))
    X = np.eye(n)
    for s in range(N):
        X = L.g_theta(flow, sm.A, X, T / N, c)
        # the BF16x6 products are float32-accurate; each step adds ~1e-7 relative
        assert P.rel_fro(host(U[s + 1]), X) < 1e-6, s
    plan.close()


def test_mixed_learned_solve_matches_oracle_taylor_parareal():
    """BF16x6 fine sweep with the float64 learned coarse propagator (Taylor constant network):
    the oracle's Taylor-4 parareal iteration count (+-1) and its result to the mixed accuracy.
    (A BF16 coarse propagator is not smooth below ~2^-24 |G|, which floors dx near 2e-8 on this
    family; the float64 coarse arithmetic removes that floor.)"""
    cuda_or_fail()
    n, T, N, J, tol = 256, 1.0, 16, 16, 1e-7
    sm = inputs.sym_matrix(n, "inv_wide", 81)
    Gt = lambda _n, x: L.g_theta(0, sm.A, x, T / N, [1, 1, 1, 1])
    F = lambda _n, x: P.rk4(0, x, sm.A, T / N, J)
    ro = P.parareal_generic(np.eye(n), N, Gt, F, N, tol)
    for refine in (0, 2):
        plan = fa.Plan(n, 0, T, N, J, fine_dtype="bf16x6", coarse_dtype="f64", max_iters=N,
                       tol=tol, coarse_kind=fa.FA_COARSE_LEARNED, refine_steps=refine)
        plan.set_learned(L.to_blob(_const_params([1.0, 1.0, 1.0, 1.0])))
        X, rep = plan.solve(dev(sm.A))
        assert rep["converged"] and abs(rep["iters"] - ro.iterations) <= 1, (rep["iters"], ro.iterations)
        assert np.all(host(plan.learned_coefs()) == 1.0)
        if refine == 0:
            # the BF16x6 fine propagator's rounding (~2^-24 per stage) grows with the flow's
            # sensitivity as X grows ~30x here: ~3e-5 against the float64 fine solution
            assert P.rel_fro(host(X), ro.U[N]) < 1e-4
        else:
            # two float64 Newton-Schulz steps reach A^{-1} itself
            inv = (sm.Q / sm.lam[None, :]) @ sm.Q.T
            assert P.rel_fro(host(X), inv) < 1e-10
        plan.close()


def test_trained_weights_beat_euler_on_held_out_matrices():
    """The committed network (trained by the library's kernels on n in [256, 1024]) on held-out
    matrices of the family at N = 64, J = 64: fewer iterations than forward Euler and no more
    than the Taylor-4 control, the same refined result."""
    cuda_or_fail()
    from paper_1505_07959_gb300 import learned as LG
    params = np.fromfile(LG.DEFAULT_WEIGHTS, dtype=np.float32)
    assert params.size == fa.FA_MLP_PARAMS and np.all(np.isfinite(params))
    res = LG.evaluate(params, ns=(256,), seeds=range(200000, 200003), N=64, J=64, tol=1e-8,
                      dtype="bf16x6", coarse_dtype="f64", refine_steps=2)
    it = {k: np.mean([r["iters"] for r in res[k]]) for k in res}
    assert it["learned"] < it["euler"], it
    assert it["learned"] <= it["taylor4"], it
    for k in res:
        for r in res[k]:
            assert r["converged"] and r["err"] < 1e-12 and r["g_fallback_iter"] == 0, (k, r)


def test_trained_weights_at_the_top_of_the_training_range():
    """The committed network at n = 1024 (the top of its training range), two held-out seeds,
    N = 64, J = 64: fewer parareal iterations than forward Euler and no more than the Taylor-4
    control on average, every result refined to float64 accuracy."""
    cuda_or_fail()
    from paper_1505_07959_gb300 import learned as LG
    params = np.fromfile(LG.DEFAULT_WEIGHTS, dtype=np.float32)
    res = LG.evaluate(params, ns=(1024,), seeds=range(200010, 200012), N=64, J=64, tol=1e-8,
                      dtype="bf16x6", coarse_dtype="f64", refine_steps=2)
    it = {k: np.mean([r["iters"] for r in res[k]]) for k in res}
    print(f"learned G at n = 1024: mean iterations {it}")
    assert it["learned"] < it["euler"], it
    assert it["learned"] <= it["taylor4"], it
    for k in res:
        for r in res[k]:
            assert r["converged"] and r["err"] < 1e-12, (k, r)
