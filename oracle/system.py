"""The discrete space-time system of Eqs. (fullysystem)/(axb) with Dirichlet data.

Reading A6 (the paper does not say how Dirichlet data enter): symmetric
elimination. Rows and columns of constrained DOFs are zeroed (kept in the
pattern), the diagonal is +1 for displacement and -1 for pressure DOFs (so A and
S = tau C + beta L stay SPD and AA keeps its saddle-point signs), the right-hand
side of a constrained row is +g_D(t_n) (u) or -g_D(t_n) (p), and free rows carry
the lifting -AA[:, D] g_D(t_n) + A'[:, D] g_D(t_{n-1}). The same elimination is
applied to A'. Step n solves AA x_n = A' x_{n-1} + F[n], n = 1..N_t.
"""
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .mesh import structured_mesh
from .fem import assemble, stabilisation_beta
from .problems import dirichlet_dofs, dirichlet_values, initial_state, load_vector, mandel_plate_penalty


@dataclass
class BiotSystem:
    case: object
    coords: np.ndarray
    tris: np.ndarray
    AA: sp.csr_matrix        # eliminated saddle-point matrix
    Ap: sp.csr_matrix        # eliminated previous-step matrix A'
    AA_full: sp.csr_matrix   # before elimination
    Ap_full: sp.csr_matrix
    F: np.ndarray            # [N_t + 1, N_dof]; row 0 unused (zero)
    x0: np.ndarray           # [N_dof]
    dir_dofs: np.ndarray
    beta: float

    @property
    def n_dof(self):
        return self.AA.shape[0]

    @property
    def u_idx(self):
        return np.sort(np.concatenate([np.arange(0, self.n_dof, 3), np.arange(1, self.n_dof, 3)]))

    @property
    def p_idx(self):
        return np.arange(2, self.n_dof, 3)

    def dscale(self):
        """d = |diag AA|^(-1/2), the Jacobi equilibration of reading A8."""
        return 1.0 / np.sqrt(np.abs(self.AA.diagonal()))


def eliminate(M, dofs, diag_values):
    """Zero rows/columns `dofs` of M (keeping the pattern) and set the diagonal."""
    M = M.tocsr(copy=True)
    mask = np.zeros(M.shape[0], dtype=bool)
    mask[dofs] = True
    rows = np.repeat(np.arange(M.shape[0]), np.diff(M.indptr))
    kill = mask[rows] | mask[M.indices]
    M.data[kill] = 0.0
    if diag_values is not None:
        dv = dict(zip(dofs.tolist(), diag_values.tolist()))
        for k in np.nonzero(kill & (rows == M.indices))[0]:
            M.data[k] = dv[rows[k]]
    return M


def add_in_pattern(M, E):
    """M + E with M's stored pattern kept (explicit zeros included): every entry of E must be a
    stored position of M (scipy's sum would drop M's explicit zeros)."""
    M = M.tocsr(copy=True)
    E = E.tocoo()
    for r, c, v in zip(E.row, E.col, E.data):
        lo, hi = M.indptr[r], M.indptr[r + 1]
        k = lo + np.searchsorted(M.indices[lo:hi], c)
        assert k < hi and M.indices[k] == c, (r, c)
        M.data[k] += v
    return M


def build_system(case, beta=None) -> BiotSystem:
    """The eliminated system of `case`. beta (optional) overrides the stabilisation factor
    of the case's own mesh size (the coarse levels of the multigrid keep the fine one)."""
    coords, tris = structured_mesh(case.n, case.Lx, case.Ly)
    h = max(case.Lx, case.Ly) / case.n
    if beta is None:
        beta = stabilisation_beta(case.E, case.nu, h, case.beta_mode)
    AA_full, Ap_full = assemble(coords, tris, case.E, case.nu, case.alpha,
                                case.kappa_elem(), case.tau, beta)
    if case.problem == "mandel":  # the rigid plate (reading A19): a penalty on the top row's u_y
        AA_full = add_in_pattern(AA_full, mandel_plate_penalty(case))
    n_dof = AA_full.shape[0]
    D = dirichlet_dofs(case)
    sign = np.where(D % 3 == 2, -1.0, 1.0)
    AA = eliminate(AA_full, D, sign)
    Ap = eliminate(Ap_full, D, None)
    F = np.zeros((case.n_t + 1, n_dof))
    free = np.ones(n_dof, dtype=bool)
    free[D] = False
    gD_prev = dirichlet_values(case, coords, D, 0.0)
    for n in range(1, case.n_t + 1):
        t = n * case.tau
        gD = dirichlet_values(case, coords, D, t)
        lift_now = np.zeros(n_dof)
        lift_now[D] = gD
        lift_prev = np.zeros(n_dof)
        lift_prev[D] = gD_prev
        f = load_vector(case, coords, tris, t) - AA_full @ lift_now + Ap_full @ lift_prev
        f[~free] = sign * gD
        F[n] = f
        gD_prev = gD
    x0 = initial_state(case, coords)
    return BiotSystem(case, coords, tris, AA, Ap, AA_full, Ap_full, F, x0, D, beta)
