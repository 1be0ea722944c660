"""Multigrid block solves (biot_set_inner_solver) against the oracle's V-cycle.

With BIOT_INNER_GMG the block solves of P1/P2 are V-cycles on the nested meshes n, n/2, ...
(Chebyshev smoothing with node-block Jacobi, restriction P^T, linear prolongation, Galerkin
coarse operators, exact band solve on the coarsest level). The oracle restates the same
cycle in plain NumPy/SciPy (oracle/gmg.py, pinned in tests/test_oracle_gmg.py), so a P^{-1}
apply must match it element by element: to rounding in FP64 (1e-10 relative per field; the
two differ only in summation order, in the power-method estimates that set the Chebyshev
interval and in the coarsest solve, band Cholesky against sparse LU) and to FP32 rounding
in the reduced-precision mode. Converged solves with multigrid block solves must still reach
backward Euler (1e-10 in FP64, 1e-8 with FP32 sweeps and the FP64 refinement).
"""
import numpy as np
import pytest

import workloads as W
from oracle.gmg import GMGPreconditioner
from oracle.solvers import field_rel_errors, seq_solve
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


def apply_both(case, kind, levels, smooth, cycles, precision, ncols=5, seed=0):
    s = build_system(case)
    P = GMGPreconditioner(s, case, kind, levels=levels, cycles=cycles, pre=smooth, post=smooth)
    vin = np.random.default_rng(seed).standard_normal((ncols, s.n_dof))
    with biot.Context(case, stream=torch.cuda.current_stream(), precision=precision, precond=kind,
                      gmg=dict(levels=levels, cycles=cycles, smooth=smooth)) as c:
        info = c.info
        z = biot.biot_precond_apply(c.ctx, vin)
    worst = 0.0
    for k in range(ncols):
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), P.apply(vin[k])[None].repeat(2, 0))
        worst = max(worst, eu, ep)
    return worst, info, P


@pytest.mark.parametrize("kind", ["diag", "tri"])
@pytest.mark.parametrize("levels,smooth,cycles", [(2, 2, 1), (3, 1, 1), (3, 3, 2)])
def test_gmg_apply_matches_oracle_fp64(kind, levels, smooth, cycles):
    case = W.terzaghi_small().with_(n=32, n_t=7, precond=kind)
    err, info, P = apply_both(case, kind, levels, smooth, cycles, "fp64")
    assert info.inner == biot.BIOT_INNER_GMG and info.gmg_levels == levels
    assert info.gmg_lam_u == pytest.approx(P.mg.u[0].lam, rel=1e-12)
    assert info.gmg_lam_p == pytest.approx(P.mg.p[0].lam, rel=1e-12)
    assert err < 1e-10, err


@pytest.mark.parametrize("problem", ["mms", "barry_mercer"])
def test_gmg_apply_other_boundary_conditions(problem):
    # all-Dirichlet (manufactured) and tangential-only (Barry & Mercer) boundaries, lognormal K
    case = W.terzaghi_small().with_(n=32, n_t=5, problem=problem, kappa=W.lognormal_kappa(32, -2.0, 1.0, 0.1, 9),
                                    E=2.0, nu=0.4, tau=0.05, precond="tri")
    err, info, _ = apply_both(case, "tri", 3, 2, 1, "fp64", ncols=4)
    assert err < 1e-10, err


def test_gmg_apply_ragged_window_and_levels_auto():
    # 13 columns (not a multiple of the 16-byte chunk) and the automatic depth (64 -> 32 -> 16)
    case = W.large_1024().with_(n=64, n_t=13, kappa=W.lognormal_kappa(64, -6.0, 2.0, 0.1, 4321))
    err, info, _ = apply_both(case, "tri", 3, 2, 1, "fp64", ncols=13)
    assert info.gmg_levels == 3
    assert err < 1e-10, err


@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_gmg_apply_fp32(kind):
    case = W.terzaghi_small().with_(n=32, n_t=6, precond=kind)
    err, _, _ = apply_both(case, kind, 3, 2, 1, "fp32", ncols=6)
    assert err < 1e-4, err


@pytest.mark.parametrize("precision,bound", [("fp64", 1e-10), ("fp32", 1e-8)])
@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_pint_with_gmg_converges_to_backward_euler(precision, bound, kind):
    case = W.terzaghi_small().with_(n=32, n_t=12, precond=kind)
    ref = seq_solve(build_system(case))
    with biot.Context(case, stream=torch.cuda.current_stream(), precision=precision,
                      gmg=dict(levels=0, cycles=1, smooth=2)) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    assert st == biot.BIOT_OK and rel <= 1e-12
    eu, ep = field_rel_errors(X, ref)
    assert eu < bound and ep < bound, (eu, ep)


def test_gmg_stress_material_fp32_reaches_1e8():
    # nu = 0.49, lognormal sigma 2: the material of the 1024^2 stress workload
    k = W.lognormal_kappa(64, -6.0, 2.0, 0.1, 4321)
    case = W.large_1024().with_(n=64, n_t=10, kappa=k, n_iter=30)
    ref = seq_solve(build_system(case))
    with biot.Context(case, stream=torch.cuda.current_stream(), precision="fp32",
                      gmg=dict(levels=0, cycles=1, smooth=2)) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-11, 20000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, ref)
    print(f"GMG FP32 stress material 64^2: {sweeps} sweeps, residual {rel:.1e}, errors {eu:.1e} {ep:.1e}")
    assert st == biot.BIOT_OK
    assert eu < 1e-8 and ep < 1e-8, (eu, ep)


def test_gmg_rejects_odd_or_small_meshes_and_switches_back():
    case = W.terzaghi_small().with_(n=15, n_t=3)
    with biot.Context(case) as c:
        with pytest.raises(biot.BiotError) as e:
            biot.biot_set_inner_solver(c.ctx, biot.BIOT_INNER_GMG, 0, 1, 2)
        assert e.value.status == biot.BIOT_E_INVALID
    case = W.terzaghi_small().with_(n=32, n_t=3)
    vin = np.random.default_rng(2).standard_normal((2, case.n_dof))
    with biot.Context(case, gmg=dict(levels=2, cycles=1, smooth=2)) as c:
        zg = biot.biot_precond_apply(c.ctx, vin)
        biot.biot_set_inner_solver(c.ctx, biot.BIOT_INNER_EXACT, 0, 1, 1)
        biot.biot_precond_setup(c.ctx, biot.BIOT_PRECOND_DIAG)
        assert c.info.gmg_levels == 0
        ze = biot.biot_precond_apply(c.ctx, vin)
    from oracle.solvers import BlockPreconditioner
    s = build_system(case)
    Pe = BlockPreconditioner(s, "diag")
    assert max(field_rel_errors(ze[0][None].repeat(2, 0), Pe.apply(vin[0])[None].repeat(2, 0))) < 1e-9
    # the V-cycle is an approximation of the exact solve, not the exact solve
    assert max(field_rel_errors(zg[0][None].repeat(2, 0), ze[0][None].repeat(2, 0))) > 1e-6
