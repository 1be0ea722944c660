"""Closed-form solutions and error norms used to pin the oracle.

Terzaghi's one-dimensional consolidation (the problem the model generalises,
Sec. 1): with roller sides the 2D solution of the Terzaghi column is the 1D one.
For incompressible constituents (no storage term, as in Eq. biotsys2), a load
sigma0 applied at t = 0+ on the drained top y = L of a column with an impervious
fixed bottom gives the undrained pressure p0 = sigma0 / alpha and

    p(y, t)   = p0 sum_k 4 (-1)^k / ((2k+1) pi) cos((2k+1) pi y / (2L)) exp(-(2k+1)^2 pi^2 c_v t / (4 L^2)),
    u_y(y, t) = (alpha int_0^y p dy' - sigma0 y) / (lambda + 2 mu),   c_v = K (lambda + 2 mu) / alpha^2.
"""
import numpy as np

from .fem import lame


def terzaghi(y, t, E, nu, alpha, K, load=1.0, L=1.0, terms=400):
    """(p, u_y) of the Terzaghi column at heights y and time t > 0."""
    lam, mu = lame(E, nu)
    M = lam + 2.0 * mu
    cv = K * M / alpha ** 2
    p0 = load / alpha
    y = np.asarray(y, dtype=np.float64)
    p = np.zeros_like(y)
    ip = np.zeros_like(y)
    for k in range(terms):
        m = (2 * k + 1) * np.pi / (2.0 * L)
        decay = np.exp(-m * m * cv * t)
        coef = 4.0 * (-1) ** k / ((2 * k + 1) * np.pi) * p0 * decay
        p += coef * np.cos(m * y)
        ip += coef * np.sin(m * y) / m
    uy = (alpha * ip - load * y) / M
    return p, uy


# 7-point degree-5 rule on the reference triangle (Radon): barycentric points, weights sum to 1.
_A1, _B1 = 0.059715871789770, 0.470142064105115
_A2, _B2 = 0.797426985353087, 0.101286507323456
QUAD7_BARY = np.array([
    [1 / 3, 1 / 3, 1 / 3],
    [_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
    [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2],
])
QUAD7_W = np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3)


def l2_error_p1(coords, tris, nodal, exact_fn):
    """|v_h - v|_{L2(Omega)} for a P1 nodal field v_h and a callable exact_fn(x, y)."""
    p = coords[tris]
    det = (p[:, 1, 0] - p[:, 0, 0]) * (p[:, 2, 1] - p[:, 0, 1]) - (p[:, 2, 0] - p[:, 0, 0]) * (p[:, 1, 1] - p[:, 0, 1])
    area = 0.5 * np.abs(det)
    vals = nodal[tris]
    total = np.zeros(tris.shape[0])
    for q in range(QUAD7_W.shape[0]):
        lb = QUAD7_BARY[q]
        x = lb[0] * p[:, 0, 0] + lb[1] * p[:, 1, 0] + lb[2] * p[:, 2, 0]
        y = lb[0] * p[:, 0, 1] + lb[1] * p[:, 1, 1] + lb[2] * p[:, 2, 1]
        vh = lb[0] * vals[:, 0] + lb[1] * vals[:, 1] + lb[2] * vals[:, 2]
        total += QUAD7_W[q] * (vh - exact_fn(x, y)) ** 2
    return float(np.sqrt(np.sum(total * area)))


def mandel_pressure(x, t, E, nu, K, F=1.0, a=1.0, terms=200):
    """Pressure of Mandel's problem (the analytic series the paper cites for Sec. 4.3) for
    alpha = 1 and no storage (Skempton B = 1):

        p(x, t) = 2 F B (1 + nu_u) / (3 a) sum_i sin(al_i) / (al_i - sin(al_i) cos(al_i))
                  (cos(al_i x / a) - cos(al_i)) exp(-al_i^2 c t / a^2),

    al_i the positive roots of tan(al) = (1 - nu) / (nu_u - nu) al (bracketed one per branch of
    tan and found by bisection), c = 2 K B^2 G (1 - nu) (1 + nu_u)^2 / (9 (1 - nu_u) (nu_u - nu)),
    G = E / (2 (1 + nu)). At t -> 0+ it tends to the undrained p0 = F B (1 + nu_u) / (3 a)."""
    from scipy.optimize import brentq
    B = 1.0
    nu_u = (3 * nu + B * (1 - 2 * nu)) / (3 - B * (1 - 2 * nu))
    G = E / (2 * (1 + nu))
    c = 2 * K * B ** 2 * G * (1 - nu) * (1 + nu_u) ** 2 / (9 * (1 - nu_u) * (nu_u - nu))
    r = (1 - nu) / (nu_u - nu)
    f = lambda al: np.sin(al) - r * al * np.cos(al)
    roots = []
    i = 0
    while len(roots) < terms:
        lo, hi = max(1e-9, (i - 0.5) * np.pi + 1e-12), (i + 0.5) * np.pi - 1e-12
        if f(lo) * f(hi) < 0:
            roots.append(brentq(f, lo, hi, xtol=1e-15))
        i += 1
    al = np.array(roots)
    x = np.asarray(x, dtype=np.float64)
    coef = np.sin(al) / (al - np.sin(al) * np.cos(al)) * np.exp(-al ** 2 * c * t / a ** 2)
    return 2 * F * B * (1 + nu_u) / (3 * a) * ((np.cos(np.outer(x, al) / a) - np.cos(al)) @ coef)
