"""Geometric multigrid for the preconditioner's blocks A and S (test infrastructure only).

Sec. 3.1 defines P1 and P2 through solves with the elasticity block A and the approximate
Schur complement S = tau C + beta L, and leaves open how those solves are done. Sec. 4 builds
its meshes by joining edge midpoints, so the uniform meshes of sizes n, n/2, n/4, ... are
nested: the coarse "/"-split mesh refined by midpoints is the fine "/"-split mesh, and the
coarse P1 space is a subspace of the fine one. This module restates, plainly, the V-cycle the
library runs as its inexact alternative to the exact block solves (reading A16):

* Levels l = 0 .. L-1 with n_l = n / 2^l. Level l's matrices are the assembled, eliminated
  blocks of the same problem on the n_l mesh with the element permeability averaged over the
  four fine children of each coarse triangle and the fine level's beta. For P1 elements on
  nested meshes this is the Galerkin product P^T M P exactly: the coarse basis gradients are
  constant on a coarse triangle, so sum_e K_e |e| grad phi_i . grad phi_j over its children is
  |E| mean(K) grad phi_i . grad phi_j; A's coefficients and beta L are constant.
* Prolongation P: linear interpolation of the coarse nodal values (fine node (2I, 2J) takes
  coarse (I, J); a fine node at the midpoint of a coarse edge the mean of its two ends, the
  "/" diagonal included). Restriction R = P^T, with the coarse Dirichlet rows set to zero.
* Smoother: Chebyshev iteration on M^{-1} K (Dirichlet rows, identity rows decoupled from the
  rest, solved exactly: x = b there), M the node-block diagonal of K (2 x 2 blocks of A,
  the diagonal of S), on the interval [lam / alpha, 1.1 lam], lam from `power_iters` steps
  of the power method on M^{-1} K from the checkerboard vector (-1)^(i + j) in every field.
  Step 0 from x = 0: d = M^{-1} b / theta, x = d. Step k >= 1 (also the first step of the
  post-smoothing, with c1 = 0, c2 = 1 / theta): s = M^{-1} (b - K x), d = c1 d + c2 s, x += d,
  with theta = (hi + lo) / 2, delta = (hi - lo) / 2, sigma = theta / delta, rho_0 = 1 / sigma,
  rho_k = 1 / (2 sigma - rho_{k-1}), c1 = rho_k rho_{k-1}, c2 = 2 rho_k / delta.
* V-cycle on level l < L-1: `pre` smoothing steps from zero, r = b - K x, coarse right-hand
  side R r, V-cycle on level l + 1, x += P x_c, `post` smoothing steps. The coarsest level
  is solved exactly (sparse LU).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .system import build_system


def coarse_kappa(kappa_e, n):
    """Per-element permeability of the n/2 mesh: the mean over the four children.

    Coarse cell (I, J) covers fine cells (2I + a, 2J + b), a, b in {0, 1}; its lower
    triangle holds the lower triangles of fine cells (2I, 2J), (2I+1, 2J), (2I+1, 2J+1) and
    the upper one of (2I+1, 2J); its upper triangle the upper ones of (2I, 2J), (2I, 2J+1),
    (2I+1, 2J+1) and the lower one of (2I, 2J+1)."""
    assert n % 2 == 0
    k = np.asarray(kappa_e, dtype=np.float64).reshape(n, n, 2)   # [j][i][lower, upper]
    nc = n // 2
    out = np.zeros((nc, nc, 2))
    for J in range(nc):
        for I in range(nc):
            j, i = 2 * J, 2 * I
            out[J, I, 0] = (k[j, i, 0] + k[j, i + 1, 0] + k[j + 1, i + 1, 0] + k[j, i + 1, 1]) / 4.0
            out[J, I, 1] = (k[j, i, 1] + k[j + 1, i, 1] + k[j + 1, i + 1, 1] + k[j + 1, i, 0]) / 4.0
    return out.reshape(-1)


def prolongation(nc):
    """Nodal linear interpolation from the nc x nc mesh to the 2nc x 2nc mesh (sparse)."""
    nf = 2 * nc
    rows, cols, vals = [], [], []
    cx = nc + 1
    for j in range(nf + 1):
        for i in range(nf + 1):
            r = j * (nf + 1) + i
            if i % 2 == 0 and j % 2 == 0:
                src = [((i // 2), (j // 2))]
            elif j % 2 == 0:
                src = [((i - 1) // 2, j // 2), ((i + 1) // 2, j // 2)]
            elif i % 2 == 0:
                src = [(i // 2, (j - 1) // 2), (i // 2, (j + 1) // 2)]
            else:  # midpoint of the "/" diagonal of coarse cell ((i-1)/2, (j-1)/2)
                src = [((i - 1) // 2, (j - 1) // 2), ((i + 1) // 2, (j + 1) // 2)]
            for (I, J) in src:
                rows.append(r)
                cols.append(J * cx + I)
                vals.append(1.0 / len(src))
    return sp.csr_matrix((vals, (rows, cols)), shape=((nf + 1) ** 2, cx * cx))


def _checkerboard(n, d):
    i = np.arange(n + 1)
    s = (-1.0) ** (i[None, :] + i[:, None])
    return np.repeat(s.reshape(-1), d)


class _Level:
    def __init__(self, K, d, n, dir_mask, alpha, power_iters):
        self.K = K.tocsr()
        self.d = d
        self.n = n
        self.dir = dir_mask
        N = K.shape[0]
        # node-block diagonal of K and its inverse
        blocks = np.zeros((N // d, d, d))
        for a in range(d):
            for b in range(d):
                blocks[:, a, b] = K[np.arange(a, N, d), np.arange(b, N, d)].A1
        self.Minv = np.linalg.inv(blocks)
        x = _checkerboard(n, d)
        lam = 0.0
        for _ in range(power_iters):
            x = x / np.linalg.norm(x)
            y = self.minv(self.K @ x)
            lam = float(np.linalg.norm(y))
            x = y
        self.lam = lam
        self.hi = 1.1 * lam
        self.lo = lam / alpha

    def minv(self, v):
        d = self.d
        return np.einsum("nab,nb->na", self.Minv, v.reshape(-1, d)).reshape(-1)

    def chebyshev(self, b, x, steps):
        """`steps` Chebyshev steps on K x = b from x (None: from zero)."""
        theta = 0.5 * (self.hi + self.lo)
        delta = 0.5 * (self.hi - self.lo)
        sigma = theta / delta
        rho = 1.0 / sigma
        dvec = None
        for k in range(steps):
            if k == 0:
                s = self.minv(b if x is None else b - self.K @ x)
                dvec = s / theta
                x = dvec.copy() if x is None else x + dvec
                # Dirichlet rows are identity rows, decoupled from the rest: solved exactly
                x[self.dir] = b[self.dir]
                dvec[self.dir] = 0.0
            else:
                rho_new = 1.0 / (2.0 * sigma - rho)
                s = self.minv(b - self.K @ x)
                dvec = rho_new * rho * dvec + (2.0 * rho_new / delta) * s
                rho = rho_new
                x = x + dvec
        return x


class GMG:
    """V-cycles for A (block 'u', 2 DOFs per node, ordering 2 v + f) and S (block 'p')."""

    def __init__(self, case, levels, pre=2, post=2, alpha=8.0, power_iters=20):
        assert case.n % (1 << (levels - 1)) == 0, "n must be divisible by 2^(levels - 1)"
        fine = build_system(case.with_(n_t=1))
        beta = fine.beta
        self.pre, self.post = pre, post
        self.u, self.p = [], []
        self.P = []
        kappa = case.kappa_elem()
        for l in range(levels):
            n_l = case.n >> l
            if l == 0:
                s = fine
            else:
                kappa = coarse_kappa(kappa, n_l * 2)
                s = build_system(case.with_(n=n_l, kappa=kappa, n_t=1), beta=beta)
            AA = s.AA.tocsr()
            ui, pi = s.u_idx, s.p_idx
            dmask = np.zeros(s.n_dof, dtype=bool)
            dmask[s.dir_dofs] = True
            self.u.append(_Level(AA[ui][:, ui], 2, n_l, dmask[ui], alpha, power_iters))
            self.p.append(_Level(-AA[pi][:, pi], 1, n_l, dmask[pi], alpha, power_iters))
            if l > 0:
                self.P.append(prolongation(n_l))
        self.lu_u = spla.splu(self.u[-1].K.tocsc())
        self.lu_p = spla.splu(self.p[-1].K.tocsc())

    def _prolong(self, l, xc, d):
        """Level l + 1 -> level l, per field."""
        P = self.P[l]
        out = np.zeros(P.shape[0] * d)
        for f in range(d):
            out[f::d] = P @ xc[f::d]
        return out

    def _restrict(self, l, r, d, coarse_dir):
        P = self.P[l]
        out = np.zeros(P.shape[1] * d)
        for f in range(d):
            out[f::d] = P.T @ r[f::d]
        out[coarse_dir] = 0.0
        return out

    def vcycle(self, block, b, l=0):
        levels = self.u if block == "u" else self.p
        d = 2 if block == "u" else 1
        L = levels[l]
        if l == len(levels) - 1:
            return (self.lu_u if block == "u" else self.lu_p).solve(b)
        x = L.chebyshev(b, None, self.pre)
        r = b - L.K @ x
        bc = self._restrict(l, r, d, levels[l + 1].dir)
        x = x + self._prolong(l, self.vcycle(block, bc, l + 1), d)
        return L.chebyshev(b, x, self.post)

    def solve(self, block, b, cycles=1):
        """`cycles` V-cycles from zero: x_{k+1} = x_k + V(b - K x_k)."""
        K = (self.u if block == "u" else self.p)[0].K
        x = self.vcycle(block, b)
        for _ in range(cycles - 1):
            x = x + self.vcycle(block, b - K @ x)
        return x


class GMGPreconditioner:
    """P1^{-1} / P2^{-1} (Eqs. p1, p2) with the block solves replaced by GMG V-cycles."""

    def __init__(self, sys, case, kind, levels, cycles=1, **kw):
        self.kind = kind
        self.cycles = cycles
        self.u = sys.u_idx
        self.p = sys.p_idx
        self.Bt = sys.AA.tocsr()[self.p][:, self.u]
        self.mg = GMG(case, levels, **kw)

    def apply(self, v):
        z = np.zeros_like(v)
        zu = self.mg.solve("u", v[self.u], self.cycles)
        if self.kind == "tri":
            zp = self.mg.solve("p", self.Bt @ zu - v[self.p], self.cycles)
        else:
            zp = -self.mg.solve("p", v[self.p], self.cycles)
        z[self.u] = zu
        z[self.p] = zp
        return z
