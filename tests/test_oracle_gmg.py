"""Pins of the oracle's geometric multigrid (oracle/gmg.py), independent of the GPU path.

The multigrid V-cycle is the library's inexact alternative to the exact block solves of
P1/P2 (Sec. 3.1 leaves the block solves open; Sec. 4's meshes come from joining edge
midpoints, so they are nested). What fixes each piece:

* prolongation: linear interpolation reproduces linear fields exactly and every row sums to 1;
* coarse operators: for P1 on nested meshes, assembling the coarse mesh with the children's
  mean permeability and the fine beta IS the Galerkin product P^T K P (checked entry by entry
  on the free DOFs against the fine matrix, lognormal permeability);
* smoother: m Chebyshev steps from zero leave the error T_m((theta - M^{-1}K)/delta) / T_m(sigma)
  times the initial one (checked through the eigen-decomposition of M^{-1/2} K M^{-1/2});
* power method: its estimate is at most the largest eigenvalue and within a few percent of it;
* the whole preconditioner: converged PinT with V-cycle block solves equals backward Euler.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import workloads as W
from oracle.gmg import GMG, GMGPreconditioner, coarse_kappa, prolongation
from oracle.solvers import field_rel_errors, pint_sweeps, seq_solve
from oracle.system import build_system


def test_prolongation_reproduces_linear_fields():
    nc = 6
    P = prolongation(nc)
    np.testing.assert_allclose(np.asarray(P.sum(axis=1)).ravel(), 1.0, rtol=0, atol=1e-15)
    xc = np.linspace(0, 1, nc + 1)
    Xc, Yc = np.meshgrid(xc, xc)           # node j (nc+1) + i at (x_i, y_j)
    xf = np.linspace(0, 1, 2 * nc + 1)
    Xf, Yf = np.meshgrid(xf, xf)
    for f in (lambda x, y: 1.0 + 0 * x, lambda x, y: 2 * x - 3 * y + 0.5, lambda x, y: x + y):
        np.testing.assert_allclose(P @ f(Xc, Yc).ravel(), f(Xf, Yf).ravel(), rtol=0, atol=1e-14)
    # a quadratic is not reproduced at the "/" diagonal midpoints: the interpolation is linear
    q = lambda x, y: x * y
    assert np.abs(P @ q(Xc, Yc).ravel() - q(Xf, Yf).ravel()).max() > 1e-3


def test_coarse_kappa_is_the_mean_of_the_children():
    n = 8
    k = W.lognormal_kappa(n, -6.0, 2.0, 0.1, 7)
    kc = coarse_kappa(k, n)
    assert kc.shape == (2 * (n // 2) ** 2,)
    # total permeability * area is preserved (every coarse triangle has four equal children)
    assert kc.sum() * 4 == pytest.approx(k.sum(), rel=1e-14)
    np.testing.assert_allclose(coarse_kappa(np.full(2 * n * n, 3.0), n), 3.0, rtol=0, atol=0)


@pytest.mark.parametrize("problem", ["terzaghi", "mms", "barry_mercer"])
def test_coarse_operators_are_galerkin_products(problem):
    n = 8
    k = W.lognormal_kappa(n, -6.0, 1.5, 0.1, 11)
    case = W.terzaghi_small().with_(n=n, n_t=1, problem=problem, kappa=k, nu=0.35)
    fine = build_system(case)
    coarse = build_system(case.with_(n=n // 2, kappa=coarse_kappa(k, n)), beta=fine.beta)
    P = prolongation(n // 2)
    for blk, d in (("u", 2), ("p", 1)):
        idx_f = fine.u_idx if blk == "u" else fine.p_idx
        idx_c = coarse.u_idx if blk == "u" else coarse.p_idx
        Kf = fine.AA.tocsr()[idx_f][:, idx_f]
        Kc = coarse.AA.tocsr()[idx_c][:, idx_c]
        Pb = sp.kron(P, sp.identity(d)).tocsr()
        free_f = np.ones(Kf.shape[0], bool)
        free_c = np.ones(Kc.shape[0], bool)
        dof_f = np.setdiff1d(np.arange(fine.n_dof), fine.dir_dofs)
        dof_c = np.setdiff1d(np.arange(coarse.n_dof), coarse.dir_dofs)
        free_f[:] = np.isin(idx_f, dof_f)
        free_c[:] = np.isin(idx_c, dof_c)
        Pff = Pb[free_f][:, free_c]
        G = (Pff.T @ Kf[free_f][:, free_f] @ Pff).toarray()
        Kcc = Kc[free_c][:, free_c].toarray()
        assert np.abs(G - Kcc).max() <= 1e-12 * np.abs(Kcc).max(), blk
        # no fine Dirichlet DOF receives anything from a free coarse DOF
        assert abs(Pb[~free_f][:, free_c]).max() == 0.0


def test_chebyshev_steps_follow_the_chebyshev_polynomial():
    case = W.terzaghi_small().with_(n=8, n_t=1)
    mg = GMG(case, levels=2, pre=3, post=3)
    for L in (mg.u[0], mg.p[0]):
        free = ~L.dir
        K = L.K.toarray()[np.ix_(free, free)]
        N = L.K.shape[0]
        Minv = np.zeros((N, N))
        d = L.d
        for v in range(N // d):
            Minv[v * d:(v + 1) * d, v * d:(v + 1) * d] = L.Minv[v]
        Mf = Minv[np.ix_(free, free)]
        rng = np.random.default_rng(3)
        xs = np.zeros(N)
        xs[free] = rng.standard_normal(free.sum())
        b = L.K @ xs
        theta = 0.5 * (L.hi + L.lo)
        delta = 0.5 * (L.hi - L.lo)
        sigma = theta / delta
        # M^{-1} K = M^{-1/2} (M^{-1/2} K M^{-1/2}) M^{1/2}; Mf is SPD (inverse of SPD blocks)
        w, Q = np.linalg.eigh(Mf)
        Mh = Q @ np.diag(np.sqrt(w)) @ Q.T          # Mf^{1/2} = M^{-1/2}
        lam, U = np.linalg.eigh(Mh @ K @ Mh)
        for m in (1, 2, 3):
            x = L.chebyshev(b, None, m)
            e = xs - x
            Tm = np.cos(m * np.arccos(np.clip((theta - lam) / delta, -1, 1))) * (np.abs((theta - lam) / delta) <= 1) \
                + np.cosh(m * np.arccosh(np.maximum(np.abs((theta - lam) / delta), 1))) * \
                np.sign((theta - lam) / delta) ** m * (np.abs((theta - lam) / delta) > 1)
            Tsig = np.cosh(m * np.arccosh(sigma))
            # error in the M^{-1/2}-scaled variables: y = M^{-1/2, inverse} e = Mh^{-1} e
            y0 = np.linalg.solve(Mh, xs[free])
            ypred = U @ ((Tm / Tsig) * (U.T @ y0))
            np.testing.assert_allclose(np.linalg.solve(Mh, e[free]), ypred, rtol=0, atol=1e-10 * np.abs(y0).max())
            assert np.all(e[~free] == 0.0)


def test_power_method_estimate_bounds_the_spectrum():
    case = W.large_1024().with_(n=16, n_t=1, kappa=W.lognormal_kappa(16, -6.0, 2.0, 0.1, 4321))
    mg = GMG(case, levels=2)
    for L in (mg.u[0], mg.p[0]):
        N = L.K.shape[0]
        Minv = sp.block_diag([sp.csr_matrix(m) for m in L.Minv])
        lam_true = np.max(np.abs(np.linalg.eigvals((Minv @ L.K).toarray())))
        assert L.lam <= lam_true * (1 + 1e-12)
        assert L.lam >= 0.95 * lam_true


@pytest.mark.parametrize("kind", ["tri", "diag"])
def test_vcycle_contracts_and_pint_with_vcycles_reaches_backward_euler(kind):
    case = W.terzaghi_small().with_(n=16, n_t=6, precond=kind)
    s = build_system(case)
    P = GMGPreconditioner(s, case, kind, levels=2)
    rng = np.random.default_rng(1)
    for blk in ("u", "p"):
        K = (P.mg.u if blk == "u" else P.mg.p)[0].K
        dirm = (P.mg.u if blk == "u" else P.mg.p)[0].dir
        xs = rng.standard_normal(K.shape[0])
        xs[dirm] = 0.0
        x = P.mg.vcycle(blk, K @ xs)
        assert np.linalg.norm(xs - x) < 0.6 * np.linalg.norm(xs), blk
        # two cycles are one cycle applied to the remaining residual
        x2 = P.mg.solve(blk, K @ xs, cycles=2)
        np.testing.assert_allclose(x2, x + P.mg.vcycle(blk, K @ (xs - x)), rtol=0, atol=1e-12 * np.abs(xs).max())
    X, nsw, conv, _ = pint_sweeps(s, P, 10, mode="tol", tol=1e-12)
    assert conv
    eu, ep = field_rel_errors(X, seq_solve(s))
    assert eu < 1e-10 and ep < 1e-10
