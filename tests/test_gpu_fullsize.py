"""Parity at the full benchmark sizes, in the launch configuration the bench times.

256 x 256 mesh (198,147 DOF), N_t = W = 256, FP64, P2, automatic strips and tuned variants:
the bench workload. The oracle assembles it in about 10 s and factors its blocks by sparse LU in
about 4 s, so the tests compare, element by element,
* the CSR pattern (bit for bit), every matrix value, A'_pp, the right-hand sides and x_0,
* the window residual of a random state on sampled steps (every DOF row of those steps),
* P^{-1} applied to the full window (256 columns, the sweep's launch shape) on sampled columns,
with the oracle. The lognormal workload (sigma 1, P1) is checked the same way in FP32 on sampled
columns. The 1024 x 1024 stress mesh (3.15M DOF, nu = 0.49, lognormal kappa sigma 2, P1) is
beyond the oracle's seconds; there a property that holds at any size is checked instead: the
exact block solves invert the assembled blocks (A z_u = v_u, S z_p = B^T z_u - v_p with
S = -AA_pp), computed on the host in FP64 with the library's CSR.
"""
import numpy as np
import pytest

import workloads as W
from oracle import fem
from oracle.mesh import structured_mesh
from oracle.solvers import BlockPreconditioner, field_rel_errors, step_residual
from oracle.system import build_system

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_2310_10430_gb300 import biot  # noqa: E402
from paper_2310_10430_gb300 import build as B  # noqa: E402

B.build()


@pytest.fixture(scope="module")
def bench_case():
    case = W.terzaghi_256("diag")
    return case, build_system(case)


@pytest.fixture(scope="module")
def bench_ctx(bench_case):
    case, _ = bench_case
    c = biot.Context(case, window=case.n_t, precision="fp64")
    t = biot.biot_tune(c.ctx, None)
    yield c, t
    c.close()


def row_scale(vals, rowptr):
    """max |value| of each entry's row, per entry"""
    a = np.abs(vals)
    starts = rowptr[:-1]
    nonempty = rowptr[1:] > starts
    mx = np.zeros(len(starts))
    mx[nonempty] = np.maximum.reduceat(a, starts[nonempty])
    return np.repeat(np.maximum(mx, 1e-300), np.diff(rowptr))


def test_bench_workload_assembly(bench_case, bench_ctx):
    case, s = bench_case
    c, t = bench_ctx
    assert t.strips == 14  # the bench's automatic choice at 256^2 in FP64
    rowptr, col, val, ap = biot.biot_get_csr(c.ctx)
    F = biot.biot_get_rhs(c.ctx)
    x0 = biot.biot_get_solution(c.ctx, 0)
    coords, tris = structured_mesh(case.n)
    rp, cc = fem.csr_pattern(tris, 3 * coords.shape[0])
    assert np.array_equal(rowptr.astype(np.int64), rp) and np.array_equal(col.astype(np.int64), cc)
    AA = s.AA.tocsr()
    assert np.max(np.abs(val - AA.data) / row_scale(AA.data, AA.indptr)) <= 1e-13
    Ap = s.Ap.tocsr()
    ref_ap = np.concatenate([Ap.data[Ap.indptr[3 * v + 2] + 2:Ap.indptr[3 * v + 3]:3] for v in range(case.n_nodes)])
    assert np.abs(ap - ref_ap).max() <= 1e-13 * np.abs(ref_ap).max()
    for f in range(3):
        fs = max(np.abs(s.F[:, f::3]).max(), 1e-300)
        assert np.abs(F[:, f::3] - s.F[:, f::3]).max() <= 1e-13 * fs, f
    assert np.abs(x0 - s.x0).max() <= 1e-14 * max(np.abs(s.x0).max(), 1.0)


def test_bench_workload_residual_sampled_steps(bench_case, bench_ctx):
    case, s = bench_case
    c, _ = bench_ctx
    rng = np.random.default_rng(17)
    X = rng.standard_normal((case.n_t + 1, s.n_dof)) * np.where(np.arange(s.n_dof) % 3 == 2, 1.0, 1e-4)
    biot.biot_set_state(c.ctx, 0, case.n_t, X)
    R = biot.biot_get_residual(c.ctx, 1, case.n_t)
    rel = biot.biot_residual_norms(c.ctx, 1, case.n_t)
    d = s.dscale()
    absA, absAp = abs(s.AA), abs(s.Ap)
    for n in (1, 2, 97, 128, 255, 256):
        r, b = step_residual(s, X, n)
        bound = absA @ np.abs(X[n]) + absAp @ np.abs(X[n - 1]) + np.abs(s.F[n])
        err = np.abs(R[n - 1] - r) / (bound + 1e-300)
        assert err.max() <= 1e-13, (n, err.max())
        assert rel[n - 1] == pytest.approx(np.linalg.norm(d * r) / np.linalg.norm(d * b), rel=1e-12)


def test_bench_workload_apply_sampled_columns(bench_case, bench_ctx):
    case, s = bench_case
    c, _ = bench_ctx
    P = BlockPreconditioner(s, "diag")
    vin = np.random.default_rng(5).standard_normal((case.n_t, s.n_dof))
    z = biot.biot_precond_apply(c.ctx, vin)  # the whole window: 128 column pairs, as in the sweep
    for k in (0, 1, 130, 254, 255):
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), P.apply(vin[k])[None].repeat(2, 0))
        assert eu < 1e-9 and ep < 1e-9, (k, eu, ep)


def test_lognormal_workload_fp32_apply_sampled_columns():
    case = W.lognormal_256()
    s = build_system(case)
    P = BlockPreconditioner(s, case.precond)
    vin = np.random.default_rng(8).standard_normal((case.n_t, s.n_dof))
    with biot.Context(case, precision="fp32") as c:
        biot.biot_tune(c.ctx, None)
        z = biot.biot_precond_apply(c.ctx, vin)
    for k in (0, 77, 255):
        eu, ep = field_rel_errors(z[k][None].repeat(2, 0), P.apply(vin[k])[None].repeat(2, 0))
        assert eu < 1e-3 and ep < 1e-3, (k, eu, ep)   # FP32 factors: cond(block) * 2^-24


def test_stress_mesh_block_solves_invert_the_blocks():
    # the 1024^2 stress mesh and material with a short window (FP64 sweeps: every block solve
    # exact to FP64 rounding; no natural-order factors above n = 512; dense-block separators)
    sp = pytest.importorskip("scipy.sparse")
    case = W.large_1024().with_(n_t=4)
    vin = np.random.default_rng(6).standard_normal((4, case.n_dof))
    with biot.Context(case, precision="fp64") as c:
        t = biot.biot_tune(c.ctx, None)
        z = biot.biot_precond_apply(c.ctx, vin)
        rowptr, col, val, _ = biot.biot_get_csr(c.ctx)
    assert t.strips == 28  # min((n + 10) / 18, sqrt((n + 1) / 1.31)) in FP64
    K = sp.csr_matrix((val, col, rowptr), shape=(len(rowptr) - 1,) * 2)
    nd = K.shape[0]
    u = np.flatnonzero(np.arange(nd) % 3 != 2)
    p = np.arange(2, nd, 3)
    Kp = K[p]
    Auu, Spp, Bt = K[u][:, u], -Kp[:, p], Kp[:, u]
    for k in range(vin.shape[0]):
        ru = np.linalg.norm(Auu @ z[k, u] - vin[k, u]) / np.linalg.norm(vin[k, u])
        rhs = Bt @ z[k, u] - vin[k, p]
        rp = np.linalg.norm(Spp @ z[k, p] - rhs) / np.linalg.norm(rhs)
        assert ru < 1e-10 and rp < 1e-10, (k, ru, rp)
