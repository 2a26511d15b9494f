"""fa_fine_sweep and fa_coarse_sweep against the oracle's fine_sweep / coarse_sweep, slice by
slice, for every flow, on ragged sizes that span several tiles."""
import numpy as np
import pytest

from gpu_helpers import MIXED, cuda_or_fail, dev, fa, host, rel, torch
from oracle import parareal as orc
from paper_1505_07959_gb300 import inputs

pytestmark = pytest.mark.gpu

# Horizons keep one Euler substep per slice stable for every flow (for the square-root flow
# dT = 1 keeps the coarse iterates positive definite; with dT = 2, I + 2(A - I) has negative
# eigenvalues and the flow X' = A - X^2 blows up from there, in the oracle as well).
FLOWS = [(fa.FA_FLOW_INV, "inv", 1.0), (fa.FA_FLOW_EXP, "exp", 1.0), (fa.FA_FLOW_SQRT, "sqrt", 2.0)]
# Error of the mixed fine sweep relative to ||F||_F: J steps of size h each add
# h ||Fl'|| times the product error of the dtype; over one slice (J h = dT) and
# with ||Fl'|| <= 4 on these spectra that is ~4 dT eps_d, plus the float32
# rounding of stage operands (~2^-24 per step, absorbed by the double-float state).
SWEEP_TOL = {"bf16": 2e-2, "bf16x3": 5e-5, "bf16x4": 1e-5, "bf16x6": 1e-6}


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    cuda_or_fail()


def _slices(sm, flow, T, N, rng):
    """N starting points: the oracle's Step-0 coarse iterates, perturbed (general inputs)."""
    U, _ = orc.coarse_sweep(sm.A, flow, T, N, 1, np.eye(sm.A.shape[0]))
    out = []
    for n in range(N):
        E = rng.standard_normal(sm.A.shape) * 1e-3
        out.append(U[n] + E)
    return np.stack(out)


@pytest.mark.parametrize("n", [16, 64, 130])
@pytest.mark.parametrize("flow,kind,T", FLOWS)
def test_fine_sweep_f64(n, flow, kind, T):
    sm = inputs.sym_matrix(n, kind, 5)
    N, J = 3, 4
    U = _slices(sm, flow, T, N, np.random.default_rng(n))
    plan = fa.Plan(n, flow, T, N, fine_steps=J, fine_dtype="f64")
    plan.set_matrix(dev(sm.A))
    F = host(plan.fine_sweep(dev(U)))
    ref = orc.fine_sweep(sm.A, flow, T, N, J, list(U))
    for b in range(N):
        e = rel(F[b], ref[b])
        assert e < 1e-12, (b, e)


@pytest.mark.parametrize("dtype", MIXED)
@pytest.mark.parametrize("n", [64, 200, 300])
@pytest.mark.parametrize("flow,kind,T", FLOWS)
def test_fine_sweep_mixed(dtype, n, flow, kind, T):
    sm = inputs.sym_matrix(n, kind, 6)
    N, J = 2, 4
    U = _slices(sm, flow, T, N, np.random.default_rng(n + 1))
    plan = fa.Plan(n, flow, T, N, fine_steps=J, fine_dtype=dtype)
    plan.set_matrix(dev(sm.A))
    F = host(plan.fine_sweep(dev(U)))
    ref = orc.fine_sweep(sm.A, flow, T, N, J, list(U))
    errs = [rel(F[b], ref[b]) for b in range(N)]
    print(f"fine sweep {dtype} n={n} flow={kind}: {['%.2e' % e for e in errs]}")
    assert max(errs) < SWEEP_TOL[dtype], errs


@pytest.mark.parametrize("n", [96, 101])
@pytest.mark.parametrize("m", [1, 3])
@pytest.mark.parametrize("dtype", ["f64", "bf16x6"])
@pytest.mark.parametrize("flow,kind,T", FLOWS)
def test_coarse_sweep(n, m, dtype, flow, kind, T):
    """Step 0 and the corrected sweep with norms.  n = 101 leaves a 5-column tail in the last
    32-column chunk (the epilogues' element-wise path) and padded operand rows (ldp = 104)."""
    N = 5
    sm = inputs.sym_matrix(n, kind, 7)
    rng = np.random.default_rng(3)
    D = rng.standard_normal((N, n, n)) * 1e-3
    Uold = np.stack([np.eye(n)] + [np.eye(n) + 0.01 * rng.standard_normal((n, n)) for _ in range(N)])
    plan = fa.Plan(n, flow, T, N, fine_steps=2, coarse_steps=m, fine_dtype=dtype)
    plan.set_matrix(dev(sm.A))
    # Step 0 (no correction)
    U0g, G0g, _ = plan.coarse_sweep(dev(np.eye(n)))
    U0, G0 = orc.coarse_sweep(sm.A, flow, T, N, m, np.eye(n))
    # float64: summation order only.  Mixed: each product element is rounded to float32
    # (2^-24) before the float64 Euler update, so G carries ~dt 2^-24 relative error per
    # substep; over N*m <= 15 substeps with dt ||Fl'|| <= 1 that stays below 1e-6.
    tol = 1e-13 if dtype == "f64" else 1e-6
    for k in range(N + 1):
        assert rel(host(U0g)[k], U0[k]) < tol
    for k in range(N):
        assert rel(host(G0g)[k], G0[k]) < tol
    # with the correction D and the norms against Uold
    Ug, Gg, normsg = plan.coarse_sweep(dev(np.eye(n)), D=dev(D), Uold=dev(Uold))
    U1, G1 = orc.coarse_sweep(sm.A, flow, T, N, m, np.eye(n), list(D))
    Ug, normsg = host(Ug), host(normsg)
    for k in range(N + 1):
        assert rel(Ug[k], U1[k]) < tol, k
    for k in range(N):
        d2 = orc.fro(U1[k + 1] - Uold[k + 1]) ** 2
        v2 = orc.fro(U1[k + 1]) ** 2
        # float64: only summation order differs; mixed: V itself carries ~1e-8 relative error,
        # which the difference V - Uold (~1e-2 of V) magnifies 100-fold in d2.
        assert abs(normsg[k, 0] - d2) <= (1e-10 if dtype == "f64" else 1e-4) * d2
        assert abs(normsg[k, 1] - v2) <= (1e-12 if dtype == "f64" else 1e-6) * v2


@pytest.mark.parametrize("flow,kind,T", FLOWS)
def test_coarse_sweep_bf16x4_row_epilogue(flow, kind, T):
    """BF16x4's term pairs are not symmetric (three terms of the left factor, two of the right),
    so its Euler launches keep the untransposed product and the row-per-thread epilogue: that
    path against the oracle on a ragged size, Step 0 and the corrected sweep with norms."""
    n, N, m = 101, 4, 1
    sm = inputs.sym_matrix(n, kind, 8)
    rng = np.random.default_rng(4)
    D = rng.standard_normal((N, n, n)) * 1e-3
    Uold = np.stack([np.eye(n)] + [np.eye(n) + 0.01 * rng.standard_normal((n, n)) for _ in range(N)])
    plan = fa.Plan(n, flow, T, N, fine_steps=2, coarse_steps=m, fine_dtype="bf16x4")
    plan.set_matrix(dev(sm.A))
    Ug, Gg, normsg = plan.coarse_sweep(dev(np.eye(n)), D=dev(D), Uold=dev(Uold))
    U1, G1 = orc.coarse_sweep(sm.A, flow, T, N, m, np.eye(n), list(D))
    Ug, Gg, normsg = host(Ug), host(Gg), host(normsg)
    plan.close()
    # the BF16x4 product error (~4e-6 of the product, test_gpu_12) times dt ||Fl'|| per step
    for k in range(N + 1):
        assert rel(Ug[k], U1[k]) < 3e-5, k
    for k in range(N):
        assert rel(Gg[k], G1[k]) < 3e-5, k
        d2 = orc.fro(U1[k + 1] - Uold[k + 1]) ** 2
        v2 = orc.fro(U1[k + 1]) ** 2
        assert abs(normsg[k, 0] - d2) <= 5e-3 * d2
        assert abs(normsg[k, 1] - v2) <= 1e-4 * v2
