"""Reduced-precision sweeps with FP64 iterative refinement, against the FP64 oracle.

BIOT_FP32: the PinT sweep (residual, P1/P2 block solves, FGMRES) runs in FP32 on the
correction system AA d_n - A' d_{n-1} = r_n of the FP64 space-time residual; x += d
in FP64 until the FP64 residual meets tol. Target: per-field relative error <= 1e-8
against the exact backward-Euler solution (the oracle's seq_solve).
BIOT_BF16VAL_FP32ACC: the same with the sweep's matrix values stored in BF16
(accumulated in FP32). BF16 values perturb AA by ~2^-9 relative; the refinement
converges only while cond * 2^-9 < 1, so its reached error is reported, not assumed.
"""
import numpy as np
import pytest

import workloads as W
from oracle.solvers import BlockPreconditioner, field_rel_errors, seq_solve
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


@pytest.mark.parametrize("kind", ["tri", "diag"])
def test_fp32_preconditioner_apply(kind):
    case = W.terzaghi_small().with_(precond=kind, n=12, n_t=4)
    s = build_system(case)
    P = BlockPreconditioner(s, kind)
    vin = np.random.default_rng(2).standard_normal((3, s.n_dof))
    with biot.Context(case, precision="fp32") as c:
        z = biot.biot_precond_apply(c.ctx, vin)
    for k in range(3):
        ref = P.apply(vin[k])
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), ref[None].repeat(2, 0))
        assert eu < 1e-3 and ep < 1e-3, (eu, ep)   # FP32 factors: cond(block) * 2^-24


@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_fp32_refinement_reaches_1e8(kind):
    case = W.terzaghi_small().with_(precond=kind)
    Xs = seq_solve(build_system(case))
    with biot.Context(case, precision="fp32") as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and rel <= 1e-12
    assert eu <= 1e-8 and ep <= 1e-8, (eu, ep)


def test_fp32_refinement_lognormal_mms():
    case = W.terzaghi_small().with_(n=10, problem="mms", E=2.0, nu=0.4, kappa=0.3, tau=0.05, n_t=19, precond="tri")
    Xs = seq_solve(build_system(case))
    with biot.Context(case, precision="fp32", window=6) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and eu <= 1e-8 and ep <= 1e-8, (eu, ep)


def test_bf16_values_refinement_reports_its_accuracy():
    case = W.terzaghi_small().with_(precond="tri")
    Xs = seq_solve(build_system(case))
    with biot.Context(case, precision="bf16") as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 20000, allow_not_converged=True)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
        rel_check = biot.biot_residual_norms(c.ctx, 1, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    print(f"bf16 values: status {biot.STATUS_NAMES[st]}, sweeps {sweeps}, space-time residual {rel:.2e}, "
          f"error u {eu:.2e} p {ep:.2e}")
    assert st in (biot.BIOT_OK, biot.BIOT_E_NOT_CONVERGED)
    assert np.all(np.isfinite(X)) and np.all(np.isfinite(rel_check))
    if st == biot.BIOT_OK:
        assert eu <= 1e-8 and ep <= 1e-8, (eu, ep)
