"""Boundary data, loads and exact solutions of the three test families.

Terzaghi column (reading A9; the paper's model, Sec. 2.1, with its standard
consolidation set-up): unit square, traction (0, -load) on the top for every
t_n >= tau, drained top (p = 0), fixed bottom (u = 0), roller sides (u_x = 0),
no flux elsewhere, initial state x0 = 0.

Trigonometric manufactured solution (Sec. 4.1): u1 = u2 = p =
cos(t) cos(3 pi x) cos(3 pi y), Dirichlet data for u and p on all sides, initial
state the exact solution at t = 0. The printed body force f matches the PDE; the
printed source g carries a sign error in its first term (it must be symmetric
under x <-> y because the solution is). Reading A3: both sources are derived
here from the PDE (biotsys1)-(biotsys2) for the stated solution.

Mandel's problem (Sec. 4.3, reading A19): the quarter domain [0, a] x [0, b] under a rigid,
frictionless plate pressed down with the total force F (the quarter's share); x = a drained and
traction-free (p = 0), x = 0 and y = 0 symmetry planes (u_x = 0, resp. u_y = 0, no flux), the
top impervious with its vertical displacement constant along x. The constraint is imposed by
a penalty: k_p (u_y(i+1) - u_y(i))^2 / 2 for consecutive top nodes with k_p = 1e4 (lambda + 2 mu),
and the force as the uniform traction (0, -F / a) on the top (under the constraint only its
total matters). Initial state: the undrained response printed in Sec. 4.3, p0 = F B (1 + nu_u)
/ (3 a), u = (F nu_u x / (2 G a), -F (1 - nu_u) y / (2 G a)), with Skempton's B = 1 (alpha = 1
and no storage: incompressible constituents) and nu_u = (3 nu + B (1 - 2 nu)) / (3 - B (1 - 2 nu)).

Barry & Mercer's problem (Sec. 4.2): the domain [0, a] x [0, b] is drained on every side
(p = 0) with zero tangential displacement there (u_y = 0 on x = 0, a; u_x = 0 on y = 0, b;
the normal component is left free, traction-free in the normal direction: reading A14), a
point source g(t) = -0.5 load delta_{(x0, y0)} sin(beta t) with beta = (lambda + 2 mu) K / (a b)
at (x0, y0) = (a / 4, b / 4), no body force, x0 = 0. The source enters the pressure rows as
-tau G^n with G^n_v = phi_v(x0, y0) g(t_n): the P1 basis functions of the triangle holding
the point, evaluated there (the exact load of a Dirac delta).
"""
import numpy as np

from .mesh import boundary_nodes
from .fem import lame, p1_geometry

K3 = 3.0 * np.pi


def mms_exact(x, y, t):
    """Exact (u1, u2, p) of the trigonometric test at time t."""
    v = np.cos(t) * np.cos(K3 * x) * np.cos(K3 * y)
    return v, v, v


def mms_sources(x, y, t, lam, mu, alpha, K):
    """Body force (f1, f2) and fluid source g for the trigonometric test.

    With c = cos, s = sin of 3 pi x / 3 pi y and k = 3 pi:
      f1 = k^2 cos t [(lam + 3 mu) cx cy - (lam + mu) sx sy] - alpha k cos t sx cy
      f2 = k^2 cos t [(lam + 3 mu) cx cy - (lam + mu) sx sy] - alpha k cos t cx sy
      g  = alpha k sin t (sx cy + cx sy) + 2 K k^2 cos t cx cy
    """
    k = K3
    cx, sx = np.cos(k * x), np.sin(k * x)
    cy, sy = np.cos(k * y), np.sin(k * y)
    common = k * k * np.cos(t) * ((lam + 3 * mu) * cx * cy - (lam + mu) * sx * sy)
    f1 = common - alpha * k * np.cos(t) * sx * cy
    f2 = common - alpha * k * np.cos(t) * cx * sy
    g = alpha * k * np.sin(t) * (sx * cy + cx * sy) + 2.0 * K * k * k * np.cos(t) * cx * cy
    return f1, f2, g


def mms_f_as_printed(x, y, t, lam, mu, alpha):
    """The body force exactly as Sec. 4.1 prints it (used only to pin mms_sources)."""
    k = K3
    cx, sx = np.cos(k * x), np.sin(k * x)
    cy, sy = np.cos(k * y), np.sin(k * y)
    f1 = -k * np.cos(t) * (alpha * sx * cy - k * (lam + 3 * mu) * cx * cy + k * (lam + mu) * sx * sy)
    f2 = -k * np.cos(t) * (alpha * cx * sy - k * (lam + 3 * mu) * cx * cy + k * (lam + mu) * sx * sy)
    return f1, f2


def area_load(coords, tris, values_at):
    """Nodal load int fun * phi_a by the 3-point edge-midpoint rule (exact to degree 2).

    values_at(x, y) evaluates the source at arrays of points. Returns a nodal
    vector of length n_nodes.
    """
    area, _, _ = p1_geometry(coords, tris)
    p = coords[tris]
    out = np.zeros(coords.shape[0])
    mids = [(0, 1), (1, 2), (2, 0)]
    fm = [values_at(0.5 * (p[:, a, 0] + p[:, b, 0]), 0.5 * (p[:, a, 1] + p[:, b, 1])) for a, b in mids]
    # phi_a is 1/2 at the midpoints of the two edges through vertex a, 0 at the third.
    for a in range(3):
        s = np.zeros(tris.shape[0])
        for q, (i0, i1) in enumerate(mids):
            if a in (i0, i1):
                s += 0.5 * fm[q]
        np.add.at(out, tris[:, a], area / 3.0 * s)
    return out


def top_traction_y(n, coords, ty):
    """Nodal load int t_y phi_a ds over the top edge for a constant traction t_y."""
    top = boundary_nodes(n)["top"]
    out = np.zeros(coords.shape[0])
    for k in range(n):
        a, b = top[k], top[k + 1]
        length = coords[b, 0] - coords[a, 0]
        out[a] += 0.5 * length * ty
        out[b] += 0.5 * length * ty
    return out


def point_source_weights(n, Lx, Ly, x0, y0):
    """(nodes, weights): the P1 basis functions of the triangle holding (x0, y0), evaluated
    there. Cell (i, j) is split along its "/" diagonal into the lower triangle (i,j),
    (i+1,j), (i+1,j+1) and the upper one (i,j), (i+1,j+1), (i,j+1); with local coordinates
    (xi, eta) in the cell, the lower one holds xi >= eta."""
    hx, hy = Lx / n, Ly / n
    i = min(int(np.floor(x0 / hx)), n - 1)
    j = min(int(np.floor(y0 / hy)), n - 1)
    xi, eta = x0 / hx - i, y0 / hy - j
    nx = n + 1
    v00, v10, v11, v01 = j * nx + i, j * nx + i + 1, (j + 1) * nx + i + 1, (j + 1) * nx + i
    if xi >= eta:
        return np.array([v00, v10, v11]), np.array([1.0 - xi, xi - eta, eta])
    return np.array([v00, v11, v01]), np.array([1.0 - eta, xi, eta - xi])


def barry_mercer_beta(case):
    """beta = (lambda + 2 mu) K / (a b) of the source's sin(beta t)."""
    lam, mu = lame(case.E, case.nu)
    return (lam + 2.0 * mu) * float(case.kappa_elem()[0]) / (case.Lx * case.Ly)


def dirichlet_dofs(case):
    """Sorted array of constrained DOFs for the case's boundary-condition family."""
    sides = boundary_nodes(case.n)
    if case.problem == "terzaghi":
        d = [3 * sides["bottom"], 3 * sides["bottom"] + 1,
             3 * sides["left"], 3 * sides["right"], 3 * sides["top"] + 2]
    elif case.problem == "barry_mercer":
        nodes = np.unique(np.concatenate(list(sides.values())))
        d = [3 * sides["bottom"], 3 * sides["top"],            # u_x tangential on y = 0, b
             3 * sides["left"] + 1, 3 * sides["right"] + 1,    # u_y tangential on x = 0, a
             3 * nodes + 2]                                    # drained everywhere
    elif case.problem == "mms":
        nodes = np.unique(np.concatenate(list(sides.values())))
        d = [3 * nodes, 3 * nodes + 1, 3 * nodes + 2]
    elif case.problem == "mandel":
        d = [3 * sides["left"], 3 * sides["bottom"] + 1, 3 * sides["right"] + 2]
    else:
        raise ValueError(case.problem)
    return np.unique(np.concatenate(d))


MANDEL_PENALTY = 1e4   # k_p / (lambda + 2 mu) of the rigid-plate constraint


def mandel_undrained(case):
    """(B, nu_u, G, p0) of Mandel's undrained response (Sec. 4.3) for alpha = 1, no storage."""
    lam, mu = lame(case.E, case.nu)
    B = 1.0
    nu_u = (3 * case.nu + B * (1 - 2 * case.nu)) / (3 - B * (1 - 2 * case.nu))
    p0 = case.load * B * (1 + nu_u) / (3 * case.Lx)
    return B, nu_u, mu, p0


def mandel_plate_penalty(case):
    """Sparse n_dof x n_dof matrix of the rigid-plate penalty: for consecutive top nodes i, i+1,
    k_p [[1, -1], [-1, 1]] on their u_y DOFs (the pairs are mesh neighbours, so the pattern of AA
    already holds every entry)."""
    import scipy.sparse as sp
    lam, mu = lame(case.E, case.nu)
    kp = MANDEL_PENALTY * (lam + 2 * mu)
    top = boundary_nodes(case.n)["top"]
    rows, cols, vals = [], [], []
    for a, b in zip(top[:-1], top[1:]):
        ia, ib = 3 * a + 1, 3 * b + 1
        rows += [ia, ia, ib, ib]
        cols += [ia, ib, ia, ib]
        vals += [kp, -kp, -kp, kp]
    nd = 3 * (case.n + 1) ** 2
    return sp.csr_matrix((vals, (rows, cols)), shape=(nd, nd))


def dirichlet_values(case, coords, dofs, t):
    """Prescribed values g_D(t) at the constrained DOFs."""
    if case.problem in ("terzaghi", "barry_mercer", "mandel"):
        return np.zeros(dofs.shape[0])
    node, field = dofs // 3, dofs % 3
    u1, u2, p = mms_exact(coords[node, 0], coords[node, 1], t)
    return np.where(field == 0, u1, np.where(field == 1, u2, p))


def initial_state(case, coords):
    """x0 in node-interleaved layout."""
    x0 = np.zeros(3 * coords.shape[0])
    if case.problem == "mms":
        u1, u2, p = mms_exact(coords[:, 0], coords[:, 1], 0.0)
        x0[0::3], x0[1::3], x0[2::3] = u1, u2, p
    elif case.problem == "mandel":
        B, nu_u, G, p0 = mandel_undrained(case)
        F, a = case.load, case.Lx
        x0[0::3] = F * nu_u * coords[:, 0] / (2 * G * a)
        x0[1::3] = -F * (1 - nu_u) * coords[:, 1] / (2 * G * a)
        x0[2::3] = p0
    return x0


def load_vector(case, coords, tris, t):
    """Unconstrained right-hand side f^n = [F^n; -tau G^n] of Eq. (fullysystem) at t = t_n."""
    nn = coords.shape[0]
    out = np.zeros(3 * nn)
    if case.problem == "terzaghi":
        out[1::3] += top_traction_y(case.n, coords, -case.load)
    elif case.problem == "mandel":
        out[1::3] += top_traction_y(case.n, coords, -case.load / case.Lx)
    elif case.problem == "barry_mercer":
        nodes, w = point_source_weights(case.n, case.Lx, case.Ly, case.Lx / 4.0, case.Ly / 4.0)
        g = -0.5 * case.load * np.sin(barry_mercer_beta(case) * t)
        out[3 * nodes + 2] += -case.tau * g * w
    else:
        lam, mu = lame(case.E, case.nu)
        K = float(case.kappa_elem()[0])
        out[0::3] += area_load(coords, tris, lambda x, y: mms_sources(x, y, t, lam, mu, case.alpha, K)[0])
        out[1::3] += area_load(coords, tris, lambda x, y: mms_sources(x, y, t, lam, mu, case.alpha, K)[1])
        out[2::3] += -case.tau * area_load(coords, tris, lambda x, y: mms_sources(x, y, t, lam, mu, case.alpha, K)[2])
    return out
