"""Mandel's problem (Sec. 4.3) on the GPU against the oracle and the analytic series.

The rigid plate is the penalty of reading A19 in both the oracle and the library; the oracle's
tests pin it to the exact constraint (master-slave elimination, 1e-5) and its solution to the
cited analytic series. Here: the library's assembled matrix (penalty included), right-hand sides
and undrained initial state against the oracle's, converged PinT solves with P1 and P2 against
the oracle's backward Euler, and the pressure against the series at the paper's h = 1/32,
tau = 0.025.
"""
import numpy as np
import pytest

import workloads as W
from oracle.analytic import mandel_pressure
from oracle.solvers import field_rel_errors, seq_solve
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


def test_mandel_assembly_rhs_and_initial_state_match_oracle():
    case = W.mandel(12, 5, 0.025)
    s = build_system(case)
    with biot.Context(case, stream=torch.cuda.current_stream()) as c:
        rowptr, col, val, ap = biot.biot_get_csr(c.ctx)
        F = biot.biot_get_rhs(c.ctx)
        X0 = biot.biot_get_solution(c.ctx, 0)
    AA = s.AA.tocsr()
    AA.sort_indices()
    assert np.array_equal(rowptr, AA.indptr) and np.array_equal(col, AA.indices)
    scale = np.abs(AA.data).max()   # the penalty entries, 1e6 (lambda + 2 mu)
    assert np.abs(val - AA.data).max() <= 1e-13 * scale
    np.testing.assert_allclose(F[1:], s.F[1:], rtol=0, atol=1e-13 * np.abs(s.F).max())
    free = np.setdiff1d(np.arange(s.n_dof), s.dir_dofs)
    np.testing.assert_allclose(X0[free], s.x0[free], rtol=1e-14, atol=0)


@pytest.mark.parametrize("kind", ["tri", "diag"])
@pytest.mark.parametrize("n,strips", [(16, None), (32, 2)])
def test_mandel_pint_matches_backward_euler(kind, n, strips):
    # the plate penalty leaves the equilibrated system less well conditioned than the other
    # problems: |AA| |x| is 1e4-5e4 times |b| per step, so FP64 rounding alone leaves a residual
    # of about 3e-12 of |b| at n = 32 (step 1). Tolerance 1e-10 (FGMRES(30), the workload's cycle
    # length), well above that floor; the oracle reaches errors of 6e-12 (P2) and 2e-11 (P1)
    # against backward Euler with it. The stopping test is per step, relative to each step's
    # right-hand side f_n + M x_{n-1}; the returned residual is the space-time one relative to
    # f_ST, whose steps n > 1 hold f_n alone, so it can sit a few times above the tolerance.
    case = W.mandel(n, 24, 0.025).with_(precond=kind)
    ref = seq_solve(build_system(case))
    with biot.Context(case, stream=torch.cuda.current_stream(), strips=strips) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    assert st == biot.BIOT_OK and rel <= 1e-9
    eu, ep = field_rel_errors(X, ref)
    assert eu < 1e-10 and ep < 1e-10, (eu, ep)


def test_mandel_fp32_refinement_reaches_1e8():
    case = W.mandel(16, 20, 0.025)
    ref = seq_solve(build_system(case))
    with biot.Context(case, stream=torch.cuda.current_stream(), precision="fp32") as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-10, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, ref)
    assert st == biot.BIOT_OK and eu < 1e-8 and ep < 1e-8, (eu, ep)


def test_mandel_pressure_against_the_series_and_mandel_cryer():
    # the paper's setting: h = 1/32, tau = 0.025, P1, tol 1e-7, to t = 5 (200 steps)
    n = 32
    case = W.mandel(n, 200, 0.025)
    with biot.Context(case, stream=torch.cuda.current_stream()) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, case.tol, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    P = X[:, 2::3].reshape(-1, n + 1, n + 1)
    xs = np.linspace(0.0, 1.0, n + 1)
    for k, bound in ((40, 0.02), (200, 0.005)):
        pa = mandel_pressure(xs, k * case.tau, case.E, case.nu, 1e-6)
        assert np.abs(P[k, n // 2] - pa).max() < bound * 0.5, k
    # the centre pressure rises above the undrained 0.5 before it drains (Mandel-Cryer)
    assert P[200, 0, 0] > P[40, 0, 0] > 0.5
