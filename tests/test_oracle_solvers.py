"""Pins for the oracle's solvers (Sec. 3): Algorithm 1, P1/P2, the Krylov cycle K,
Algorithm 3 and the windowed sweep schedule.

Independent references: a dense solve of the whole space-time system (P10), the
closed-form block structure of P^{-1} AA and its spectra (P5), a brute-force
least-squares solve over an explicitly built Krylov space, the identity of
Algorithm 3 with the sweep schedule (P6), the reduction to backward Euler for a
single thread (P3, Sec. 3.2) and convergence to the sequential solution (P4).
"""
import numpy as np
import pytest

import workloads as W
from oracle.solvers import (BlockPreconditioner, field_rel_errors, fgmres_cycle, pint_alg3,
                            pint_sweeps, seq_solve, spacetime_dense_solve, spacetime_residual,
                            step_residual)
from oracle.system import build_system


def tiny(problem="terzaghi", n=3, n_t=4, **kw):
    base = dict(n=n, E=1e4, nu=0.3, alpha=1.0, kappa=1e-6, tau=1e-2, n_t=n_t, problem=problem)
    base.update(kw)
    return build_system(W.BiotCase(**base))


@pytest.mark.parametrize("problem", ["terzaghi", "mms"])
def test_seq_solve_equals_dense_spacetime_solve(problem):
    s = tiny(problem, n=3, n_t=4, E=1.0, kappa=1.0, tau=0.1)
    X = seq_solve(s)
    Xd = spacetime_dense_solve(s)
    np.testing.assert_allclose(X, Xd, rtol=1e-11, atol=1e-12 * np.abs(Xd).max())
    assert spacetime_residual(s, X) < 1e-13


def test_preconditioned_operator_block_structure():
    s = tiny(n=4, kappa=W.lognormal_kappa(4, sigma=1.0, seed=5))
    AA = s.AA.toarray()
    u, p = s.u_idx, s.p_idx
    A = AA[np.ix_(u, u)]
    B = AA[np.ix_(u, p)]
    S = -AA[np.ix_(p, p)]
    Ainv_B = np.linalg.solve(A, B)
    Sinv_Bt = np.linalg.solve(S, B.T)
    for kind in ("tri", "diag"):
        P = BlockPreconditioner(s, kind)
        PiA = np.array([P.apply(AA[:, k]) for k in range(AA.shape[0])]).T
        # Eq. p1: P1^{-1} AA = [[I, A^{-1}B], [0, I + S^{-1} B^T A^{-1} B]]
        # Eq. p2: P2^{-1} AA = [[I, A^{-1}B], [-S^{-1} B^T, I]]
        np.testing.assert_allclose(PiA[np.ix_(u, u)], np.eye(len(u)), atol=1e-10)
        np.testing.assert_allclose(PiA[np.ix_(u, p)], Ainv_B, atol=1e-10 * np.abs(Ainv_B).max())
        if kind == "tri":
            np.testing.assert_allclose(PiA[np.ix_(p, u)], 0.0, atol=1e-13 * np.abs(Sinv_Bt).max())
            np.testing.assert_allclose(PiA[np.ix_(p, p)], np.eye(len(p)) + Sinv_Bt @ Ainv_B, rtol=1e-9, atol=1e-9)
        else:
            np.testing.assert_allclose(PiA[np.ix_(p, u)], -Sinv_Bt, rtol=1e-9, atol=1e-9 * np.abs(Sinv_Bt).max())
            np.testing.assert_allclose(PiA[np.ix_(p, p)], np.eye(len(p)), atol=1e-10)
        np.testing.assert_allclose(P.dense() @ PiA, AA, atol=1e-9 * np.abs(AA).max())


def test_richardson_contraction_and_divergence():
    # Algorithm 2's update X += P^{-1}(b - AA X) is Richardson; its contraction is
    # rho1 = rho(S^{-1} B^T A^{-1} B) for P1 and sqrt(rho1) for P2 (P5) -- above 1 here.
    s = tiny(n=4, n_t=3)
    AA = s.AA.toarray()
    u, p = s.u_idx, s.p_idx
    T = np.linalg.solve(-AA[np.ix_(p, p)], AA[np.ix_(p, u)] @ np.linalg.solve(AA[np.ix_(u, u)], AA[np.ix_(u, p)]))
    rho1 = max(abs(np.linalg.eigvals(T)))
    assert rho1 > 1.0
    rhos = {}
    for kind in ("tri", "diag"):
        P = BlockPreconditioner(s, kind)
        PiA = np.array([P.apply(AA[:, k]) for k in range(AA.shape[0])]).T
        rhos[kind] = max(abs(np.linalg.eigvals(np.eye(AA.shape[0]) - PiA)))
        # literal Richardson on step 1 diverges
        b = s.F[1] + s.Ap @ s.x0
        x = np.zeros(s.n_dof)
        r0 = np.linalg.norm(b)
        for _ in range(40):
            x = x + P.apply(b - AA @ x)
        assert np.linalg.norm(b - AA @ x) > 1e3 * r0
    assert rhos["tri"] == pytest.approx(rho1, rel=1e-8)
    assert rhos["diag"] == pytest.approx(np.sqrt(rho1), rel=1e-8)


@pytest.mark.parametrize("kind", ["tri", "diag"])
@pytest.mark.parametrize("k", [1, 2, 3])
def test_fgmres_cycle_is_krylov_least_squares(kind, k):
    s = tiny("mms", n=3, n_t=2, E=1.0, kappa=1.0, tau=0.1)
    AA = s.AA.toarray()
    d = s.dscale()
    P = BlockPreconditioner(s, kind)
    rng = np.random.default_rng(k)
    x0 = rng.standard_normal(s.n_dof)
    b = rng.standard_normal(s.n_dof)
    x1, info = fgmres_cycle(s.AA, P, d, x0, b, k)
    assert info.k == k
    # brute force: right-preconditioned operator in equilibrated variables
    Pinv = np.array([P.apply(e) for e in np.eye(s.n_dof)]).T
    At = np.diag(d) @ AA @ Pinv @ np.diag(1.0 / d)
    r0 = d * (b - AA @ x0)
    Kry = np.array([np.linalg.matrix_power(At, i) @ r0 for i in range(k)]).T
    Q, _ = np.linalg.qr(Kry)
    y, *_ = np.linalg.lstsq(At @ Q, r0, rcond=None)
    x_ref = x0 + Pinv @ (Q @ y / d)
    np.testing.assert_allclose(x1, x_ref, rtol=1e-8, atol=1e-8 * np.abs(x_ref).max())
    assert np.linalg.norm(d * (b - AA @ x1)) == pytest.approx(info.est, rel=1e-6)


def test_fgmres_full_cycle_solves_and_zero_residual_is_fixed_point():
    s = tiny(n=2, n_t=1)
    d = s.dscale()
    P = BlockPreconditioner(s, "diag")
    b = s.F[1] + s.Ap @ s.x0
    x, info = fgmres_cycle(s.AA, P, d, np.zeros(s.n_dof), b, s.n_dof)
    np.testing.assert_allclose(s.AA @ x, b, atol=1e-10 * np.abs(b).max())
    x2, info2 = fgmres_cycle(s.AA, P, d, x, s.AA @ x, 5)
    assert info2.k == 0 and np.array_equal(x2, x)


@pytest.mark.parametrize("kind", ["tri", "diag"])
def test_alg3_equals_paper_mode_sweeps_bitwise(kind):
    s = tiny(n=3, n_t=5)
    P = BlockPreconditioner(s, kind)
    M = 3
    Xa = pint_alg3(s, P, M, 2)
    Xs, nsw, conv, log = pint_sweeps(s, P, 2, mode="paper", M=M)
    assert nsw == 5 + M - 1 and conv
    assert np.array_equal(Xa, Xs)
    assert [h - l + 1 for l, h in zip(log.lo, log.hi)] == [1, 2, 3, 3, 3, 2, 1]


@pytest.mark.parametrize("problem", ["terzaghi", "mms"])
def test_seq_solve_solves_every_step_to_fp64(problem):
    # Alg. 1 with an exact solve: each step's equilibrated residual is at rounding level
    s = build_system(W.terzaghi_small().with_(problem=problem, n_t=6))
    X = seq_solve(s)
    d = s.dscale()
    for n in range(1, 7):
        r, b = step_residual(s, X, n)
        assert np.linalg.norm(d * r) <= 1e-14 * np.linalg.norm(d * b)


def test_single_thread_is_backward_euler():
    # Sec. 3.2: with N_thread = 1 the inverted method is backward Euler; with an inner
    # solver that converges in one call (n_iter = N_dof) the iterates equal seq_solve.
    s = tiny(n=2, n_t=3)
    P = BlockPreconditioner(s, "tri")
    Xa = pint_alg3(s, P, 1, s.n_dof)
    X = seq_solve(s)
    np.testing.assert_allclose(Xa, X, rtol=1e-9, atol=1e-12 * np.abs(X).max())


def test_window_one_matches_sequential():
    # P3: a window of one step iterates each step to tol before the next starts
    s = build_system(W.terzaghi_small().with_(n=8, n_t=6))
    P = BlockPreconditioner(s, "diag")
    X, nsw, conv, log = pint_sweeps(s, P, 10, mode="tol", tol=1e-12, w_max=1)
    assert conv and all(h == l for l, h in zip(log.lo, log.hi))
    eu, ep = field_rel_errors(X, seq_solve(s))
    assert eu < 1e-9 and ep < 1e-9


@pytest.mark.parametrize("kind", ["tri", "diag"])
def test_pint_converges_to_sequential(kind):
    # P4: the space-time system is block lower bidiagonal with nonsingular AA, so the
    # converged PinT iterate is the backward-Euler solution.
    s = build_system(W.terzaghi_small().with_(n=8, n_t=8))
    P = BlockPreconditioner(s, kind)
    X, nsw, conv, log = pint_sweeps(s, P, 10, mode="tol", tol=1e-12)
    assert conv
    eu, ep = field_rel_errors(X, seq_solve(s))
    assert eu < 1e-10 and ep < 1e-10
    assert spacetime_residual(s, X) < 1e-11
    # tol retirement is in order and every retired step meets tol against its final predecessor
    for n in range(1, s.F.shape[0]):
        r, b = step_residual(s, X, n)
        d = s.dscale()
        assert np.linalg.norm(d * r) <= 1e-12 * np.linalg.norm(d * b) * (1 + 1e-9)


@pytest.mark.parametrize("kind", ["tri", "diag"])
def test_eager_start_converges_to_sequential_and_continues(kind):
    # The eager start (every step active from the first sweep) solves the same space-time
    # system, so it converges to the backward-Euler solution too (P4), also when it continues
    # from a state converged to 1e-6 only. Its first sweep updates every step. (It saves few
    # sweeps: A' couples each step to its predecessor at full strength, so a change made at
    # one step needs one sweep per step to reach the last, whatever the start.)
    s = build_system(W.terzaghi_small().with_(n=8, n_t=8))
    P = BlockPreconditioner(s, kind)
    X, nsw, conv, log = pint_sweeps(s, P, 10, mode="eager", tol=1e-12)
    assert conv and log.lo[0] == 1 and log.hi[0] == 8
    ref = seq_solve(s)
    eu, ep = field_rel_errors(X, ref)
    assert eu < 1e-10 and ep < 1e-10
    X6, n6, conv6, _ = pint_sweeps(s, P, 10, mode="tol", tol=1e-6)
    assert conv6 and max(field_rel_errors(X6, ref)) > 1e-9
    X12, n12, conv12, log12 = pint_sweeps(s, P, 10, mode="eager", tol=1e-12, X0=X6)
    assert conv12 and log12.hi[0] == 8
    eu, ep = field_rel_errors(X12, ref)
    assert eu < 1e-10 and ep < 1e-10
