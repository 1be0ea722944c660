"""Solvers of Sec. 3: sequential time stepping, the block preconditioners and the
inverted (parallel-in-time) time stepping.

* seq_solve: Algorithm 1 with the inner iteration replaced by an exact sparse LU
  solve of AA (factored once): x_n = AA^{-1} (A' x_{n-1} + F[n]).
* BlockPreconditioner: P1 = [[A, 0], [B^T, -S]] (Eq. p1) and P2 = [[A, 0], [0, -S]]
  (Eq. p2), S = tau C + beta L the approximate Schur complement. The block
  solves with A and S are exact (sparse LU, factored once).
* fgmres_cycle: the inner solver K(P, AA, X, b, n_iter) of Algorithm 3 (reading
  A4): one cycle of n_iter right-preconditioned flexible GMRES steps from the
  initial guess X, classical Gram-Schmidt applied twice, Givens rotations,
  minimising the Jacobi-equilibrated residual |D^{-1/2}(b - AA x)| (reading A8).
* pint_alg3: Algorithm 3 exactly as stated (outer loop over m, inner loop over n,
  b^{n,m} = A' X^{n-1,m} + f^n, X^{n,m} = K(P, AA, X^{n,m-1}, b^{n,m}, n_iter)).
* pint_sweeps: the same iteration organised as snapshot sweeps over a window of
  active time steps (reading A5), the form the GPU evaluates: at sweep w every
  active step n reads X[n-1] and X[n] from the state after sweep w-1, and step n
  becomes active at sweep n. With a fixed number M of iterations per step
  ("paper" mode) it reproduces Algorithm 3's iterates X^{n,m}, m = w - n + 1,
  operation for operation; "tol" mode retires the oldest active step once its
  predecessor is retired and its relative residual is below tol.
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

BREAKDOWN_RTOL = 1e-14


def seq_solve(sys, refine_steps=2):
    """Algorithm 1 with an exact inner solve. Returns X [N_t + 1, N_dof], X[0] = x0.

    AA mixes rows of size ~E (displacement) and ~tau K + beta (pressure); a sparse
    LU of AA itself leaves step residuals near 1e-9. The step system is therefore
    solved as D^{-1/2} AA D^{-1/2} y = D^{-1/2} b (D = |diag AA|) by sparse LU,
    x = D^{-1/2} y, followed by refine_steps steps of FP64 iterative refinement,
    which brings every step to its FP64 solution (relative residual ~1e-16).
    """
    d = sys.dscale()
    Dm = sp.diags(d)
    lu = spla.splu((Dm @ sys.AA @ Dm).tocsc())
    n_t = sys.F.shape[0] - 1
    X = np.zeros((n_t + 1, sys.n_dof))
    X[0] = sys.x0
    for n in range(1, n_t + 1):
        b = sys.Ap @ X[n - 1] + sys.F[n]
        x = d * lu.solve(d * b)
        for _ in range(refine_steps):
            x = x + d * lu.solve(d * (b - sys.AA @ x))
        X[n] = x
    return X


class BlockPreconditioner:
    """Exact application of P1^{-1} ("tri") or P2^{-1} ("diag") to a full-length vector."""

    def __init__(self, sys, kind):
        if kind not in ("tri", "diag"):
            raise ValueError(kind)
        self.kind = kind
        self.u = sys.u_idx
        self.p = sys.p_idx
        AA = sys.AA.tocsr()
        self.A = AA[self.u][:, self.u].tocsc()
        self.S = (-AA[self.p][:, self.p]).tocsc()
        self.Bt = AA[self.p][:, self.u].tocsr()
        self.A_lu = spla.splu(self.A)
        self.S_lu = spla.splu(self.S)

    def apply(self, v):
        """z = P^{-1} v. P1: z_u = A^{-1} v_u, z_p = S^{-1}(B^T z_u - v_p).
        P2: z_u = A^{-1} v_u, z_p = -S^{-1} v_p."""
        z = np.zeros_like(v)
        zu = self.A_lu.solve(v[self.u])
        if self.kind == "tri":
            zp = self.S_lu.solve(self.Bt @ zu - v[self.p])
        else:
            zp = -self.S_lu.solve(v[self.p])
        z[self.u] = zu
        z[self.p] = zp
        return z

    def dense(self):
        """The dense matrix P (for brute-force checks on tiny meshes)."""
        n = self.u.shape[0] + self.p.shape[0]
        P = np.zeros((n, n))
        P[np.ix_(self.u, self.u)] = self.A.toarray()
        P[np.ix_(self.p, self.p)] = -self.S.toarray()
        if self.kind == "tri":
            P[np.ix_(self.p, self.u)] = self.Bt.toarray()
        return P


@dataclass
class CycleInfo:
    k: int                 # Arnoldi steps taken (< n_iter after a breakdown)
    beta0: float           # |D^{-1/2} r| at the start of the cycle
    est: float             # least-squares residual estimate at the end


def fgmres_cycle(AA, P, d, x, b, n_iter, r=None):
    """One cycle of right-preconditioned FGMRES(n_iter) on the equilibrated system.

    Minimises |d * (b - AA x)| over x in x0 + span{z_0..z_{k-1}},
    z_j = P^{-1}(v_j / d), with the Arnoldi basis v_j orthonormal in the plain
    2-norm. Returns (x_new, CycleInfo).
    """
    if r is None:
        r = b - AA @ x
    rt = d * r
    beta0 = float(np.sqrt(np.dot(rt, rt)))
    if beta0 == 0.0:
        return x.copy(), CycleInfo(0, 0.0, 0.0)
    V = [rt / beta0]
    Z = []
    H = np.zeros((n_iter + 1, n_iter))
    cs = np.zeros(n_iter)
    sn = np.zeros(n_iter)
    g = np.zeros(n_iter + 1)
    g[0] = beta0
    k = 0
    for j in range(n_iter):
        z = P.apply(V[j] / d)
        w = d * (AA @ z)
        w_norm0 = float(np.sqrt(np.dot(w, w)))
        Vm = np.array(V)
        h = Vm @ w
        w = w - Vm.T @ h
        h2 = Vm @ w
        w = w - Vm.T @ h2
        h = h + h2
        hn = float(np.sqrt(np.dot(w, w)))
        H[: j + 1, j] = h
        H[j + 1, j] = hn
        Z.append(z)
        for i in range(j):
            t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
            H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
            H[i, j] = t
        den = float(np.hypot(H[j, j], H[j + 1, j]))
        if den == 0.0:
            cs[j], sn[j] = 1.0, 0.0
        else:
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
        H[j, j] = den
        H[j + 1, j] = 0.0
        g[j + 1] = -sn[j] * g[j]
        g[j] = cs[j] * g[j]
        k = j + 1
        if hn <= BREAKDOWN_RTOL * w_norm0:
            break
        V.append(w / hn)
    y = np.zeros(k)
    for i in range(k - 1, -1, -1):
        y[i] = (g[i] - np.dot(H[i, i + 1 : k], y[i + 1 : k])) / H[i, i]
    x_new = x + np.array(Z[:k]).T @ y
    return x_new, CycleInfo(k, beta0, abs(g[k]))


def step_residual(sys, X, n):
    """(r_n, b_n): b_n = F[n] + A' X[n-1], r_n = b_n - AA X[n]."""
    b = sys.F[n] + sys.Ap @ X[n - 1]
    return b - sys.AA @ X[n], b


def pint_alg3(sys, P, M, n_iter):
    """Algorithm 3 verbatim, in place: X[n] holds the latest iterate of step n.

    X^{1:N_t, 0} = 0; for m = 1..M, for n = 1..N_t:
    b^{n,m} = A' X^{n-1,m} + f^n; X^{n,m} = K(P, AA, X^{n,m-1}, b^{n,m}, n_iter).
    """
    n_t = sys.F.shape[0] - 1
    d = sys.dscale()
    X = np.zeros((n_t + 1, sys.n_dof))
    X[0] = sys.x0
    for m in range(1, M + 1):
        for n in range(1, n_t + 1):
            b = sys.Ap @ X[n - 1] + sys.F[n]
            X[n], _ = fgmres_cycle(sys.AA, P, d, X[n], b, n_iter)
    return X


@dataclass
class SweepLog:
    lo: list = field(default_factory=list)
    hi: list = field(default_factory=list)
    rel: list = field(default_factory=list)      # per active column, before the update
    retired_upto: list = field(default_factory=list)


def pint_sweeps(sys, P, n_iter, mode="tol", M=None, tol=1e-10, w_max=None, max_sweeps=100000, X0=None):
    """Windowed snapshot sweeps (reading A5). Returns (X, n_sweeps, converged, SweepLog).

    mode "paper": step n is updated at sweeps n .. n + M - 1 (M = N_thread of
    Algorithm 3), active window [max(1, w - M + 1), min(w, N_t)].
    mode "tol": active window [lo, min(w, N_t, lo + w_max - 1)]; before the
    updates of sweep w the relative residuals |d r_n| / |d b_n| of the active
    steps are formed from the snapshot; starting at lo, steps whose residual is
    <= tol retire (no update), stopping at the first that is not. The solve ends
    when every step has retired.
    mode "eager": as "tol" with every step active from the first sweep, window
    [lo, min(N_t, lo + w_max - 1)] (the start that suits a state that is already
    close to the solution, e.g. a continuation).
    X0 (optional): starting state [N_t + 1, N_dof] (row 0 is replaced by x0); zero otherwise.
    """
    n_t = sys.F.shape[0] - 1
    d = sys.dscale()
    X = np.zeros((n_t + 1, sys.n_dof)) if X0 is None else np.array(X0, dtype=np.float64)
    X[0] = sys.x0
    log = SweepLog()
    if w_max is None:
        w_max = n_t
    lo = 1
    w = 0
    while w < max_sweeps:
        if mode == "paper":
            if w >= n_t + M - 1:
                return X, w, True, log
            w += 1
            a, z = max(1, w - M + 1), min(w, n_t)
        else:
            if lo > n_t:
                return X, w, True, log
            w += 1
            a, z = lo, min(n_t if mode == "eager" else w, n_t, lo + w_max - 1)
        Xs = X.copy()
        rel = []
        res = {}
        for n in range(a, z + 1):
            r, b = step_residual(sys, Xs, n)
            rb = float(np.linalg.norm(d * b))
            rr = float(np.linalg.norm(d * r))
            rel.append(rr / rb if rb > 0 else (0.0 if rr == 0 else np.inf))
            res[n] = (r, b)
        log.lo.append(a)
        log.hi.append(z)
        log.rel.append(rel)
        if mode in ("tol", "eager"):
            while lo <= z and rel[lo - a] <= tol:
                lo += 1
            a = lo
            log.retired_upto.append(lo - 1)
        for n in range(a, z + 1):
            r, b = res[n]
            X[n], _ = fgmres_cycle(sys.AA, P, d, Xs[n], b, n_iter, r=r)
    return X, w, False, log


def spacetime_residual(sys, X):
    """Relative equilibrated space-time residual |D^{-1/2}(F - calA X)| / |D^{-1/2} F_ST|,
    F_ST[1] = F[1] + A' x0 (reading A8)."""
    n_t = sys.F.shape[0] - 1
    d = sys.dscale()
    num = 0.0
    den = 0.0
    for n in range(1, n_t + 1):
        r, _ = step_residual(sys, X, n)
        num += float(np.sum((d * r) ** 2))
        fst = sys.F[n] + (sys.Ap @ sys.x0 if n == 1 else 0.0)
        den += float(np.sum((d * fst) ** 2))
    return np.sqrt(num / den) if den > 0 else np.sqrt(num)


def spacetime_dense_solve(sys):
    """Brute force: solve the whole block-bidiagonal space-time system densely
    (tiny meshes only). Block row n: -A' x_{n-1} + AA x_n = F[n] (+ A' x0 for n = 1)."""
    n_t = sys.F.shape[0] - 1
    N = sys.n_dof
    AA = sys.AA.toarray()
    Ap = sys.Ap.toarray()
    big = np.zeros((n_t * N, n_t * N))
    rhs = np.zeros(n_t * N)
    for n in range(n_t):
        big[n * N:(n + 1) * N, n * N:(n + 1) * N] = AA
        if n > 0:
            big[n * N:(n + 1) * N, (n - 1) * N:n * N] = -Ap
        rhs[n * N:(n + 1) * N] = sys.F[n + 1]
    rhs[:N] += Ap @ sys.x0
    sol = np.linalg.solve(big, rhs)
    X = np.zeros((n_t + 1, N))
    X[0] = sys.x0
    X[1:] = sol.reshape(n_t, N)
    return X


def field_rel_errors(X, Xref):
    """Per-field relative L2 differences over all steps 1..N_t: (u, p)."""
    out = []
    for sel in (np.s_[:, 0::3], np.s_[:, 1::3]), (np.s_[:, 2::3],):
        num = sum(float(np.sum((X[1:][s] - Xref[1:][s]) ** 2)) for s in sel)
        den = sum(float(np.sum(Xref[1:][s] ** 2)) for s in sel)
        out.append(np.sqrt(num / den) if den > 0 else np.sqrt(num))
    return tuple(out)
