"""Pins for the oracle's mesh, element matrices and assembly (Sec. 2.1-2.2).

Each check fixes the oracle against something other than itself: a hand-computed
element, rigid-body and linear-field identities, the closed-form pattern size,
and the structural properties (symmetry, definiteness) the preconditioners rely on.
"""
import json
import os

import numpy as np
import pytest

import workloads as W
from oracle import fem
from oracle.mesh import structured_mesh, boundary_nodes
from oracle.problems import area_load, top_traction_y
from oracle.system import build_system

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_reference_triangle_matches_hand_computation():
    g = json.load(open(os.path.join(GOLDEN, "p1_reference_triangle.json")))
    coords = np.array(g["vertices"], dtype=float)
    tris = np.array([[0, 1, 2]])
    area, gx, gy = fem.p1_geometry(coords, tris)
    K = fem.element_elasticity(area, gx, gy, g["lam"], g["mu"])[0]
    np.testing.assert_allclose(K[0::2, 0::2], g["K_xx"], atol=1e-15)
    np.testing.assert_allclose(K[1::2, 1::2], g["K_yy"], atol=1e-15)
    np.testing.assert_allclose(K[0::2, 1::2], g["K_xy"], atol=1e-15)
    B = fem.element_coupling(area, gx, gy, g["alpha"])[0]
    for b in range(3):
        np.testing.assert_allclose(B[0::2, b], g["B_x_row"], atol=1e-15)
        np.testing.assert_allclose(B[1::2, b], g["B_y_row"], atol=1e-15)
    np.testing.assert_allclose(fem.element_laplacian(area, gx, gy)[0], g["L"], atol=1e-15)


def test_basis_gradients_reproduce_kronecker_delta():
    coords, tris = structured_mesh(3, 2.0, 1.5)
    area, gx, gy = fem.p1_geometry(coords, tris)
    assert np.all(area > 0)  # counter-clockwise
    np.testing.assert_allclose(area.sum(), 3.0, rtol=1e-14)
    p = coords[tris]
    for a in range(3):
        # phi_a(x_b) - phi_a(x_0) = grad phi_a . (x_b - x_0) must equal delta_ab - delta_a0
        for b in range(3):
            val = gx[:, a] * (p[:, b, 0] - p[:, 0, 0]) + gy[:, a] * (p[:, b, 1] - p[:, 0, 1])
            np.testing.assert_allclose(val, float(a == b) - float(a == 0), atol=1e-13)


@pytest.mark.parametrize("n", [1, 2, 5, 16])
def test_pattern_size_and_order(n):
    coords, tris = structured_mesh(n)
    rowptr, col = fem.csr_pattern(tris, 3 * coords.shape[0])
    assert rowptr[-1] == 9 * (7 * n * n + 6 * n + 1)
    for r in range(3 * coords.shape[0]):
        c = col[rowptr[r]:rowptr[r + 1]]
        assert np.all(np.diff(c) > 0)
    # a node's row holds its own and its (up to 6) mesh neighbours' DOFs
    nx = n + 1
    v = (n // 2) * nx + n // 2
    nb = sorted({v, v - 1, v + 1, v - nx, v + nx, v - nx - 1, v + nx + 1} & set(range(nx * nx))) if n >= 2 else None
    if n >= 2:
        expect = np.array([3 * m + f for m in nb for f in range(3)])
        np.testing.assert_array_equal(col[rowptr[3 * v]:rowptr[3 * v + 1]], expect)


def _full(case):
    s = build_system(case)
    return s, s.AA_full.toarray(), s.Ap_full.toarray()


def test_rigid_body_modes_and_linear_fields():
    case = W.BiotCase(n=5, E=3.0, nu=0.27, alpha=0.8, kappa=2.0, tau=0.1, n_t=1)
    s, AA, Ap = _full(case)
    x, y = s.coords[:, 0], s.coords[:, 1]
    u = np.sort(np.concatenate([np.arange(0, s.n_dof, 3), np.arange(1, s.n_dof, 3)]))
    A = AA[np.ix_(u, u)]
    for mode in ((np.ones_like(x), 0 * x), (0 * x, np.ones_like(x)), (-y, x)):
        vec = np.stack(mode, axis=1).ravel()
        np.testing.assert_allclose(A @ vec, 0.0, atol=1e-12)
    # a uniform dilatation u = (x, y) has div u = 2: B^T u = -alpha int phi_b 2
    vec = np.zeros(s.n_dof)
    vec[0::3], vec[1::3] = x, y
    Btu = (AA @ vec)[2::3]
    lumped = area_load(s.coords, s.tris, lambda a, b: np.ones_like(a))
    np.testing.assert_allclose(Btu, -2.0 * case.alpha * lumped, atol=1e-13)
    # the K-free Laplacian annihilates constants and linear fields in interior rows
    beta = s.beta
    pp = -Ap[2::3, 2::3] / beta
    np.testing.assert_allclose(pp @ np.ones_like(x), 0.0, atol=1e-12)
    interior = (x > 1e-12) & (x < 1 - 1e-12) & (y > 1e-12) & (y < 1 - 1e-12)
    np.testing.assert_allclose((pp @ (2 * x - 3 * y))[interior], 0.0, atol=1e-12)
    # AA's pp block is -(tau C + beta L), C = kappa L for constant kappa
    np.testing.assert_allclose(AA[2::3, 2::3], -(case.tau * case.kappa + beta) * pp, atol=1e-12)
    # A' and AA share B^T
    np.testing.assert_allclose(Ap[2::3][:, u], AA[2::3][:, u], atol=0)
    np.testing.assert_allclose(Ap[np.ix_(u, np.arange(s.n_dof))], 0.0, atol=0)


def test_symmetry_and_definiteness_after_elimination():
    for problem in ("terzaghi", "mms"):
        case = W.BiotCase(n=6, E=1e4, nu=0.45, alpha=1.0, kappa=W.lognormal_kappa(6, sigma=1.0, seed=3),
                          tau=1e-3, n_t=1, problem=problem)
        s = build_system(case)
        AA = s.AA.toarray()
        np.testing.assert_allclose(AA, AA.T, atol=1e-12 * np.abs(AA).max())
        u, p = s.u_idx, s.p_idx
        np.linalg.cholesky(AA[np.ix_(u, u)])           # A SPD
        np.linalg.cholesky(-AA[np.ix_(p, p)])          # S = tau C + beta L SPD
        assert np.allclose(np.diag(AA)[s.dir_dofs], np.where(s.dir_dofs % 3 == 2, -1.0, 1.0))


def test_loads_integrate_exactly():
    coords, tris = structured_mesh(7, 2.0, 3.0)
    tot = area_load(coords, tris, lambda x, y: np.ones_like(x))
    np.testing.assert_allclose(tot.sum(), 6.0, rtol=1e-14)
    # degree-2 source: int_0^2 int_0^3 x y dy dx = 2 * 4.5 = 9 (midpoint rule is exact to degree 2)
    np.testing.assert_allclose(area_load(coords, tris, lambda x, y: x * y).sum(), 9.0, rtol=1e-13)
    tr = top_traction_y(7, coords, -1.0)
    np.testing.assert_allclose(tr.sum(), -2.0, rtol=1e-14)
    top = boundary_nodes(7)["top"]
    np.testing.assert_allclose(tr[top[1:-1]], -2.0 / 7, rtol=1e-14)


def test_beta_readings():
    lam, mu = fem.lame(1e4, 0.3)
    assert fem.stabilisation_beta(1e4, 0.3, 0.5, "h2") == pytest.approx(0.25 / (4 * (lam + 2 * mu)))
    assert fem.stabilisation_beta(1e4, 0.3, 0.5, "h") == pytest.approx(0.5 / (4 * (lam + 2 * mu)))
    assert fem.stabilisation_beta(1e4, 0.3, 0.5, "none") == 0.0
    lam, mu = fem.lame(1.0, 0.25)
    assert lam == pytest.approx(0.4) and mu == pytest.approx(0.4)
