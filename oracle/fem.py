"""Stabilised P1-P1 discretisation of the two-field Biot model (Sec. 2.2).

Bilinear forms (Sec. 2.1), with reading A1 (the elasticity form carries the
lambda term of sigma(u) = 2 mu eps(u) + lambda div(u) I, which the printed
a(u, v) omits):

    a(u, v)   = int 2 mu eps(u):eps(v) + lambda div(u) div(v)   -> A
    -b(v, p)  = -alpha int p div(v)                              -> B
    c(p, q)   = int K grad p . grad q                            -> C

Backward Euler with the stabilisation (beta/K) c(dp/dt, q) (Eq. diseq1) gives,
per step, the saddle-point matrix of Eq. (fullysystem),

    AA = [[A, B], [B^T, -(tau C + beta L)]],   A' = [[0, 0], [B^T, -beta L]],

where L is the K-free P1 Laplacian, so that (beta/K) C = beta L element by
element (reading A2': exact for constant K, and the natural reading for a
per-element K).

Unknowns are node-interleaved: DOF 3 v + f with f = 0 (u_x), 1 (u_y), 2 (p).
"""
import numpy as np
import scipy.sparse as sp


def lame(E: float, nu: float):
    """Lame coefficients from Young's modulus and Poisson ratio (Sec. 2.1)."""
    lam = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    mu = E / (2.0 * (1.0 + nu))
    return lam, mu


def stabilisation_beta(E: float, nu: float, h: float, mode: str = "h2") -> float:
    """Stabilisation factor beta of Sec. 2.2.

    The paper prints beta = h / (4 (lambda + 2 mu)); the perturbation beta Laplace(dp/dt)
    is only dimensionally consistent with h^2, which is the value of the cited
    stabilised scheme. Reading A2: mode "h2" (default) uses h^2/(4(lambda+2mu)),
    mode "h" the printed formula, mode "none" switches stabilisation off.
    h is the maximal leg length of the uniform grid, 1/n on the unit square.
    """
    lam, mu = lame(E, nu)
    if mode == "h2":
        return h * h / (4.0 * (lam + 2.0 * mu))
    if mode == "h":
        return h / (4.0 * (lam + 2.0 * mu))
    if mode == "none":
        return 0.0
    raise ValueError(mode)


def p1_geometry(coords, tris):
    """Areas [E] and constant basis-function gradients gx, gy [E, 3] of P1 triangles."""
    p = coords[tris]
    x = p[:, :, 0]
    y = p[:, :, 1]
    det = (x[:, 1] - x[:, 0]) * (y[:, 2] - y[:, 0]) - (x[:, 2] - x[:, 0]) * (y[:, 1] - y[:, 0])
    area = 0.5 * det
    gx = np.stack([y[:, 1] - y[:, 2], y[:, 2] - y[:, 0], y[:, 0] - y[:, 1]], axis=1) / det[:, None]
    gy = np.stack([x[:, 2] - x[:, 1], x[:, 0] - x[:, 2], x[:, 1] - x[:, 0]], axis=1) / det[:, None]
    return area, gx, gy


def element_elasticity(area, gx, gy, lam, mu):
    """6x6 element stiffness area * Bv^T D Bv (Voigt form), local DOF order (a, d) -> 2a + d."""
    ne = area.shape[0]
    Bv = np.zeros((ne, 3, 6))
    for a in range(3):
        Bv[:, 0, 2 * a] = gx[:, a]          # eps_xx
        Bv[:, 1, 2 * a + 1] = gy[:, a]      # eps_yy
        Bv[:, 2, 2 * a] = gy[:, a]          # gamma_xy = 2 eps_xy
        Bv[:, 2, 2 * a + 1] = gx[:, a]
    D = np.array([[lam + 2 * mu, lam, 0.0], [lam, lam + 2 * mu, 0.0], [0.0, 0.0, mu]])
    return area[:, None, None] * np.einsum("eki,kl,elj->eij", Bv, D, Bv)


def element_coupling(area, gx, gy, alpha):
    """6x3 element block of B = -b(v, p): row (a, d), column b: -alpha int phi_b d_d phi_a."""
    ne = area.shape[0]
    Be = np.zeros((ne, 6, 3))
    for a in range(3):
        for b in range(3):
            Be[:, 2 * a, b] = -alpha * area / 3.0 * gx[:, a]
            Be[:, 2 * a + 1, b] = -alpha * area / 3.0 * gy[:, a]
    return Be


def element_laplacian(area, gx, gy):
    """3x3 K-free P1 Laplacian int grad phi_a . grad phi_b."""
    return area[:, None, None] * (gx[:, :, None] * gx[:, None, :] + gy[:, :, None] * gy[:, None, :])


def local_to_global(tris):
    """Global DOF indices [E, 9] for local DOF 3a + f (node a of the triangle, field f)."""
    return (3 * tris[:, :, None] + np.arange(3)[None, None, :]).reshape(-1, 9)


def element_blocks(coords, tris, E, nu, alpha, kappa_e, tau, beta):
    """9x9 element matrices of AA and A' in local DOF order 3a + f."""
    lam, mu = lame(E, nu)
    area, gx, gy = p1_geometry(coords, tris)
    Ke = element_elasticity(area, gx, gy, lam, mu)
    Be = element_coupling(area, gx, gy, alpha)
    Le = element_laplacian(area, gx, gy)
    Ce = kappa_e[:, None, None] * Le
    ne = area.shape[0]
    M = np.zeros((ne, 9, 9))
    Mp = np.zeros((ne, 9, 9))
    for a in range(3):
        for b in range(3):
            for d in range(2):
                for d2 in range(2):
                    M[:, 3 * a + d, 3 * b + d2] = Ke[:, 2 * a + d, 2 * b + d2]
                M[:, 3 * a + d, 3 * b + 2] = Be[:, 2 * a + d, b]
                M[:, 3 * b + 2, 3 * a + d] = Be[:, 2 * a + d, b]
                Mp[:, 3 * b + 2, 3 * a + d] = Be[:, 2 * a + d, b]
            M[:, 3 * a + 2, 3 * b + 2] = -(tau * Ce[:, a, b] + beta * Le[:, a, b])
            Mp[:, 3 * a + 2, 3 * b + 2] = -beta * Le[:, a, b]
    return M, Mp


def csr_pattern(tris, n_dof):
    """Sorted, duplicate-free CSR pattern (rowptr, col) of all DOF pairs that share
    a triangle (the element-coupling pattern, independent of values and BCs)."""
    g = local_to_global(tris)
    rows = np.repeat(g, 9, axis=1).ravel()
    cols = np.tile(g, (1, 9)).ravel()
    key = np.unique(rows * n_dof + cols)
    r = key // n_dof
    c = key % n_dof
    rowptr = np.zeros(n_dof + 1, dtype=np.int64)
    np.add.at(rowptr, r + 1, 1)
    rowptr = np.cumsum(rowptr)
    return rowptr, c


def assemble(coords, tris, E, nu, alpha, kappa_e, tau, beta):
    """Assemble AA and A' as scipy CSR matrices on the element-coupling pattern.

    Element contributions are added entry by entry in element order
    (np.add.at). Entries that are structurally present but numerically zero stay
    stored, so both matrices share the pattern returned by csr_pattern.
    """
    n_dof = 3 * coords.shape[0]
    M, Mp = element_blocks(coords, tris, E, nu, alpha, kappa_e, tau, beta)
    g = local_to_global(tris)
    rowptr, col = csr_pattern(tris, n_dof)
    keys = np.repeat(np.arange(n_dof), np.diff(rowptr)) * n_dof + col
    rows = np.repeat(g, 9, axis=1).ravel()
    cols = np.tile(g, (1, 9)).ravel()
    pos = np.searchsorted(keys, rows * n_dof + cols)
    assert np.array_equal(keys[pos], rows * n_dof + cols)
    out = []
    for Me in (M, Mp):
        vals = np.zeros(col.shape[0])
        np.add.at(vals, pos, Me.reshape(-1))
        out.append(sp.csr_matrix((vals, col.copy(), rowptr.copy()), shape=(n_dof, n_dof)))
    return out[0], out[1]
