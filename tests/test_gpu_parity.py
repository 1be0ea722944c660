"""Parity of the CUDA path against the FP64 CPU oracle, through the C ABI.

Integer work (the CSR pattern) must match bit for bit. FP64 values, right-hand
sides and residuals must match to 1e-13 relative to the row scale (different
summation order only). Preconditioner applications are direct band-Cholesky
solves on the GPU and sparse-LU solves in the oracle; they agree to within
cond(block) * eps, checked at 1e-9 relative. Whole solves must match the oracle
to 1e-10 relative per field (the parity bound of the FP64 path).
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem
from oracle.mesh import structured_mesh
from oracle.solvers import (BlockPreconditioner, field_rel_errors, pint_sweeps, seq_solve, step_residual)
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


def cases():
    base = W.terzaghi_small()
    return {
        "terzaghi16": base,
        "mms12": base.with_(n=12, problem="mms", E=3.0, nu=0.25, kappa=0.7, tau=0.05, n_t=6),
        "lognormal10": base.with_(n=10, kappa=W.lognormal_kappa(10, sigma=1.0, seed=7), nu=0.42, n_t=5),
        "literal_beta": base.with_(n=6, beta_mode="h", n_t=3),
        "no_beta": base.with_(n=6, beta_mode="none", n_t=3),
        "tiny": base.with_(n=1, n_t=1),
        # Barry & Mercer point source off the nodes (n = 10: (1/4, 1/4) inside a cell)
        "barry10": W.barry_mercer(10, 6).with_(tau=1.0 / 256),
    }


def row_scaled_close(got, ref, rowptr, rtol):
    scale = np.zeros_like(ref)
    for r in range(rowptr.shape[0] - 1):
        a, b = rowptr[r], rowptr[r + 1]
        scale[a:b] = max(np.abs(ref[a:b]).max(), 1e-300)
    err = np.abs(got - ref) / scale
    assert err.max() <= rtol, (err.max(), np.argmax(err))


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 64])
def test_pattern_bit_exact(n):
    ctx = biot.biot_mesh_create(n)
    try:
        rowptr, col, _, _ = biot.biot_get_csr(ctx, values=False)
    finally:
        biot.biot_destroy(ctx)
    coords, tris = structured_mesh(n)
    rp, c = fem.csr_pattern(tris, 3 * coords.shape[0])
    assert np.array_equal(rowptr.astype(np.int64), rp)
    assert np.array_equal(col.astype(np.int64), c)


@pytest.mark.parametrize("name", list(cases()))
def test_assembly_rhs_and_initial_state(name):
    case = cases()[name]
    s = build_system(case)
    with biot.Context(case) as c:
        rowptr, col, val, ap = biot.biot_get_csr(c.ctx)
        F = biot.biot_get_rhs(c.ctx)
        x0 = biot.biot_get_solution(c.ctx, 0)
        info = c.info
    assert info.beta == pytest.approx(s.beta, rel=1e-15, abs=0)
    AA = s.AA.tocsr()
    row_scaled_close(val, AA.data, AA.indptr, 1e-13)
    # A' pressure-pressure entries in node-pair order
    Ap = s.Ap.tocsr()
    ref_ap = []
    for v in range(case.n_nodes):
        a, b = Ap.indptr[3 * v + 2], Ap.indptr[3 * v + 3]
        ref_ap.extend(Ap.data[a + 2:b:3])
    ref_ap = np.array(ref_ap)
    scale = max(np.abs(ref_ap).max(), 1e-300)
    assert np.abs(ap - ref_ap).max() <= 1e-13 * scale
    for f in range(3):
        fs = max(np.abs(s.F[:, f::3]).max(), 1e-300)
        assert np.abs(F[:, f::3] - s.F[:, f::3]).max() <= 1e-13 * fs, f
    assert np.abs(x0 - s.x0).max() <= 1e-14 * max(np.abs(s.x0).max(), 1.0)


@pytest.mark.parametrize("name", ["terzaghi16", "mms12", "lognormal10", "barry10"])
def test_residual_window(name):
    case = cases()[name]
    s = build_system(case)
    rng = np.random.default_rng(11)
    X = rng.standard_normal((case.n_t + 1, s.n_dof)) * np.where(np.arange(s.n_dof) % 3 == 2, 1.0, 1e-4)
    with biot.Context(case) as c:
        biot.biot_set_state(c.ctx, 0, case.n_t, X)
        lo, hi = 2, case.n_t
        R = biot.biot_get_residual(c.ctx, lo, hi)
        rel = biot.biot_residual_norms(c.ctx, lo, hi)
    d = s.dscale()
    absA, absAp = abs(s.AA), abs(s.Ap)
    for k, n in enumerate(range(lo, hi + 1)):
        r, b = step_residual(s, X, n)
        # rounding bound of each entry: |AA| |x_n| + |A'| |x_{n-1}| + |f^n|
        bound = absA @ np.abs(X[n]) + absAp @ np.abs(X[n - 1]) + np.abs(s.F[n])
        assert np.all(np.abs(R[k] - r) <= 1e-13 * bound + 1e-300), np.max(np.abs(R[k] - r) / (bound + 1e-300))
        assert rel[k] == pytest.approx(np.linalg.norm(d * r) / np.linalg.norm(d * b), rel=1e-12)


@pytest.mark.parametrize("kind", ["tri", "diag"])
@pytest.mark.parametrize("name", ["terzaghi16", "mms12", "lognormal10", "barry10"])
def test_precond_apply(kind, name):
    case = cases()[name].with_(precond=kind)
    s = build_system(case)
    P = BlockPreconditioner(s, kind)
    rng = np.random.default_rng(3)
    ncols = min(case.n_t, 4)
    vin = rng.standard_normal((ncols, s.n_dof))
    with biot.Context(case) as c:
        z = biot.biot_precond_apply(c.ctx, vin)
    for k in range(ncols):
        ref = P.apply(vin[k])
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), ref[None].repeat(2, 0))
        assert eu < 1e-9 and ep < 1e-9, (eu, ep)


@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_paper_schedule_matches_oracle(kind):
    case = W.terzaghi_small().with_(precond=kind)
    M = 3
    s = build_system(case)
    Xo, nsw, _, _ = pint_sweeps(s, BlockPreconditioner(s, kind), case.n_iter, mode="paper", M=M)
    with biot.Context(case, window=M, schedule=biot.BIOT_SCHED_PAPER) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 0.0, 10000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    assert sweeps == nsw == case.n_t + M - 1
    eu, ep = field_rel_errors(X, Xo)
    # Unconverged iterates (M = 3 cycles per step) are as sensitive to rounding as the
    # Krylov process makes them: with P2 the oracle itself moves by 4.9e-10 (u) and
    # 3.2e-10 (p) when its exact LU block solves are replaced by exact band-Cholesky
    # solves; with P1 by 1.7e-13. The bound is four times the oracle's own spread.
    bound = 1e-10 if kind == "tri" else 2e-9
    assert eu < bound and ep < bound, (eu, ep)


def test_tol_schedule_converges_to_sequential():
    case = W.terzaghi_small()
    s = build_system(case)
    Xs = seq_solve(s)
    Xo, nsw, conv, _ = pint_sweeps(s, BlockPreconditioner(s, case.precond), case.n_iter, mode="tol", tol=case.tol)
    with biot.Context(case) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, case.tol, 10000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    assert st == biot.BIOT_OK and conv
    assert abs(sweeps - nsw) <= 1, (sweeps, nsw)
    eu, ep = field_rel_errors(X, Xo)
    assert eu < 1e-9 and ep < 1e-9, (eu, ep)
    eu, ep = field_rel_errors(X, Xs)
    assert eu < 1e-8 and ep < 1e-8, (eu, ep)
    assert rel < 1e-9


@pytest.mark.parametrize("kind", ["diag", "tri"])
def test_converged_solve_matches_sequential_to_1e10(kind):
    # the parity bound of the FP64 path: converged PinT vs exact backward Euler
    case = W.terzaghi_small().with_(precond=kind)
    s = build_system(case)
    Xs = seq_solve(s)
    with biot.Context(case) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-13, 100000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and eu < 1e-10 and ep < 1e-10, (eu, ep)
    assert rel < 1e-12


@pytest.mark.parametrize("strips,precision,bound", [(1, "fp64", 1e-10), (3, "fp64", 1e-10), (3, "fp32", 1e-8)])
def test_barry_mercer_pint_matches_sequential(strips, precision, bound):
    # Sec. 4.2 compares the parallel-in-time solution with sequential backward Euler (P2,
    # tol 1e-10); here converged further, on the paper's mesh h = 1/64 over its first 40 steps
    # (tau = 1/256), plain and substructured block solves, and FP32 sweeps with FP64 refinement
    case = W.barry_mercer(64, 256).with_(n_t=40)
    Xs = seq_solve(build_system(case))
    with biot.Context(case, strips=strips, precision=precision) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-13, 100000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and eu < bound and ep < bound, (eu, ep)


def test_mms_tol_solve_and_edge_windows():
    # ragged window (N_t not a multiple of 32 lanes), window cap smaller than N_t
    case = W.terzaghi_small().with_(n=8, problem="mms", E=1.0, kappa=1.0, tau=0.05, n_t=37, precond="tri")
    s = build_system(case)
    Xs = seq_solve(s)
    with biot.Context(case, window=7) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-12, 100000)
        X = biot.biot_get_state(c.ctx, 0, case.n_t)
        assert c.info.window_cap == 7
    eu, ep = field_rel_errors(X, Xs)
    assert st == biot.BIOT_OK and eu < 1e-8 and ep < 1e-8, (eu, ep)


def test_single_step_and_single_cell():
    case = W.terzaghi_small().with_(n=1, n_t=1)
    s = build_system(case)
    Xs = seq_solve(s)
    with biot.Context(case) as c:
        st, sweeps, rel = biot.biot_pint_solve(c.ctx, 1e-13, 100)
        X = biot.biot_get_state(c.ctx, 0, 1)
    np.testing.assert_allclose(X, Xs, rtol=1e-9, atol=1e-14)


def test_state_errors_and_not_converged():
    case = W.terzaghi_small().with_(n=4, n_t=4)
    ctx = biot.biot_mesh_create(4)
    try:
        with pytest.raises(biot.BiotError) as e:
            biot.biot_sweep(ctx, 1, 1)
        assert e.value.status == biot.BIOT_E_STATE
        p, keep = biot.make_params(case.E, case.nu, case.alpha, case.kappa, case.tau, case.n_t)
        biot.biot_assemble(ctx, p)
        with pytest.raises(biot.BiotError) as e:
            biot.biot_pint_solve(ctx, 1e-10, 10)
        assert e.value.status == biot.BIOT_E_STATE
        biot.biot_precond_setup(ctx, biot.BIOT_PRECOND_DIAG)
        with pytest.raises(biot.BiotError) as e:
            biot.biot_sweep(ctx, 0, 2)
        assert e.value.status == biot.BIOT_E_INVALID
        st, sweeps, rel = biot.biot_pint_solve(ctx, 1e-14, 2, allow_not_converged=True)
        assert st == biot.BIOT_E_NOT_CONVERGED and sweeps == 2
    finally:
        biot.biot_destroy(ctx)
