"""Seeded synthetic inputs for the parallel-in-time Biot solver.

This module is the only code shared by the CPU oracle and the CUDA path. It
holds workload descriptions (mesh size, material constants, time step, horizon,
boundary-condition family) and the seeded random permeability field; it holds
none of the method's arithmetic (no assembly, no residual, no solve).

Workloads follow the test cases of arxiv 2310.10430, Sec. 4 (unit square,
uniform right-triangle grid with h = 1/n, backward Euler with step tau) and the
synthetic configurations built on them:

* ``terzaghi``: consolidation column under a unit top load, drained top, fixed
  bottom, roller sides (the classical problem that motivates the model, Sec. 1).
* ``mms``: the trigonometric manufactured solution of Sec. 4.1,
  u1 = u2 = p = cos(t) cos(3 pi x) cos(3 pi y), Dirichlet data on all sides.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace
from typing import Optional

import numpy as np

TERZAGHI = "terzaghi"
MMS = "mms"
BARRY_MERCER = "barry_mercer"
MANDEL = "mandel"


@dataclass(frozen=True)
class BiotCase:
    """One Biot instance: geometry, material, time grid and solver options.

    ``kappa`` is either a scalar or an array with one value per triangle in the
    element order of the structured mesh (cell (i, j) -> triangles 2(j n + i)
    (lower) and 2(j n + i) + 1 (upper)).
    """

    n: int
    E: float
    nu: float
    alpha: float
    kappa: object
    tau: float
    n_t: int
    problem: str = TERZAGHI
    Lx: float = 1.0
    Ly: float = 1.0
    beta_mode: str = "h2"     # "h2": h^2/(4(lam+2mu)); "h": literal h/(4(lam+2mu)); "none": beta = 0
    precond: str = "diag"     # "diag": P2 (block diagonal); "tri": P1 (block lower triangular)
    n_iter: int = 10          # Krylov iterations per call of the inner solver K
    tol: float = 1e-10
    load: float = 1.0         # Terzaghi top load (traction (0, -load)); Barry & Mercer source amplitude 0.5 load
    name: str = ""

    def with_(self, **kw) -> "BiotCase":
        return replace(self, **kw)

    @property
    def n_nodes(self) -> int:
        return (self.n + 1) ** 2

    @property
    def n_dof(self) -> int:
        return 3 * self.n_nodes

    @property
    def n_elem(self) -> int:
        return 2 * self.n * self.n

    def kappa_elem(self) -> np.ndarray:
        """Per-element permeability as a float64 array of length 2 n^2."""
        k = self.kappa
        if np.isscalar(k):
            return np.full(self.n_elem, float(k))
        k = np.asarray(k, dtype=np.float64)
        assert k.shape == (self.n_elem,)
        return k


def element_centroids(n: int, Lx: float = 1.0, Ly: float = 1.0) -> np.ndarray:
    """Centroids [2 n^2, 2] of the structured mesh's triangles (lower, upper per cell)."""
    hx, hy = Lx / n, Ly / n
    j, i = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    i = i.ravel().astype(np.float64)
    j = j.ravel().astype(np.float64)
    lower = np.stack([(i + 2.0 / 3.0) * hx, (j + 1.0 / 3.0) * hy], axis=1)
    upper = np.stack([(i + 1.0 / 3.0) * hx, (j + 2.0 / 3.0) * hy], axis=1)
    out = np.empty((2 * n * n, 2))
    out[0::2] = lower
    out[1::2] = upper
    return out


def lognormal_kappa(n: int, mean_log10: float = -6.0, sigma: float = 1.0,
                    corr_len: float = 0.1, seed: int = 1234, n_features: int = 512,
                    Lx: float = 1.0, Ly: float = 1.0) -> np.ndarray:
    """Seeded lognormal permeability per element.

    log kappa = ln(10^mean_log10) + sigma * Z(centroid), where Z is a unit-variance
    Gaussian random field with squared-exponential covariance of length
    ``corr_len``, approximated by ``n_features`` random Fourier features
    (Rahimi-Recht): Z(x) = sqrt(2/M) sum_m cos(w_m . x + b_m), w_m ~ N(0, I/l^2),
    b_m ~ U[0, 2 pi). NumPy PCG64 with the given seed.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    w = rng.standard_normal((n_features, 2)) / corr_len
    b = rng.uniform(0.0, 2.0 * np.pi, n_features)
    c = element_centroids(n, Lx, Ly)
    # in row chunks on large meshes (the feature matrix of 1024^2 would hold 8.6 GB)
    step = 1 << 18
    z = np.concatenate([np.cos(c[i:i + step] @ w.T + b).sum(axis=1) for i in range(0, len(c), step)])
    z *= np.sqrt(2.0 / n_features)
    return np.exp(mean_log10 * np.log(10.0) + sigma * z)


# ---------------------------------------------------------------------------
# Named workloads (synthetic inputs shaped like the paper's test cases)
# ---------------------------------------------------------------------------

def terzaghi_small() -> BiotCase:
    """16x16 mesh, 867 DOF, N_t = 32, tau = 1e-2, E = 1e4, nu = 0.3, alpha = 1,
    kappa = 1e-6, Terzaghi column, block-diagonal preconditioner, tol 1e-10."""
    return BiotCase(n=16, E=1e4, nu=0.3, alpha=1.0, kappa=1e-6, tau=1e-2, n_t=32,
                    problem=TERZAGHI, precond="diag", tol=1e-10, name="terzaghi_16x16_nt32")


def terzaghi_256(precond: str = "diag") -> BiotCase:
    """256x256 mesh (66,049 nodes, 198,147 DOF), N_t = 256, tau = 1e-3, same physics."""
    return BiotCase(n=256, E=1e4, nu=0.3, alpha=1.0, kappa=1e-6, tau=1e-3, n_t=256,
                    problem=TERZAGHI, precond=precond, tol=1e-10, name="terzaghi_256x256_nt256")


def mms_256(precond: str = "tri") -> BiotCase:
    """256x256 mesh, N_t = 256, tau = 1e-3, trigonometric manufactured solution."""
    return BiotCase(n=256, E=1e4, nu=0.3, alpha=1.0, kappa=1e-6, tau=1e-3, n_t=256,
                    problem=MMS, precond=precond, tol=1e-10, name="mms_256x256_nt256")


def lognormal_256(seed: int = 1234) -> BiotCase:
    """256x256 mesh, N_t = 256, lognormal kappa (geometric mean 1e-6, sigma 1, l = 0.1)."""
    k = lognormal_kappa(256, -6.0, 1.0, 0.1, seed)
    return BiotCase(n=256, E=1e4, nu=0.3, alpha=1.0, kappa=k, tau=1e-3, n_t=256,
                    problem=TERZAGHI, precond="tri", tol=1e-8, name="lognormal_256x256_nt256")


def batched_instances(count: int = 64, seed0: int = 1000) -> list:
    """Independent instances: n drawn from multiples of 8 in [32, 192], N_t in [64, 512],
    nu in [0.2, 0.45], lognormal kappa with sigma 1.5; instance i uses seed seed0 + i."""
    out = []
    for i in range(count):
        rng = np.random.Generator(np.random.PCG64(seed0 + i))
        n = int(rng.integers(4, 25)) * 8
        n_t = int(rng.integers(64, 513))
        nu = float(rng.uniform(0.2, 0.45))
        k = lognormal_kappa(n, -6.0, 1.5, 0.1, seed0 + i)
        out.append(BiotCase(n=n, E=1e4, nu=nu, alpha=1.0, kappa=k, tau=1e-3, n_t=n_t,
                            problem=TERZAGHI, precond="tri", tol=1e-8,
                            name=f"batched_{i}_n{n}_nt{n_t}"))
    return out


def barry_mercer(n: int = 64, n_t: int = 256) -> BiotCase:
    """Barry & Mercer's point source (Sec. 4.2): unit square, h = 1/64, tau = T/256, T = 1,
    E = 1e5, nu = 0.1, K = 1e-2, source -0.5 delta_(1/4, 1/4) sin(beta t), P2, tol 1e-10."""
    return BiotCase(n=n, E=1e5, nu=0.1, alpha=1.0, kappa=1e-2, tau=1.0 / n_t, n_t=n_t,
                    problem=BARRY_MERCER, precond="diag", tol=1e-10, name=f"barry_mercer_{n}x{n}_nt{n_t}")


def large_1024() -> BiotCase:
    """1024x1024 mesh (3,151,875 DOF), N_t = 128, nu = 0.49, lognormal kappa sigma 2."""
    k = lognormal_kappa(1024, -6.0, 2.0, 0.1, 4321)
    return BiotCase(n=1024, E=1e4, nu=0.49, alpha=1.0, kappa=k, tau=1e-3, n_t=128,
                    problem=TERZAGHI, precond="tri", tol=1e-8, name="large_1024x1024_nt128")


def mandel(n: int = 32, n_t: int = 40, tau: float = 0.025) -> BiotCase:
    """Mandel's problem (Sec. 4.3): quarter domain a = b = 1, K = 1e-6, E = 1e4, nu = 0, B = 1
    (alpha = 1, no storage), F = 1, P1, tol 1e-7; the paper's plot uses h = 1/32, tau = 0.025.
    Krylov cycles of 30 steps (the restart length of the GMRES the paper uses): with the rigid
    plate, cycles of 10 stall under P2."""
    return BiotCase(n=n, E=1e4, nu=0.0, alpha=1.0, kappa=1e-6, tau=tau, n_t=n_t, problem=MANDEL,
                    precond="tri", tol=1e-7, load=1.0, n_iter=30, name=f"mandel_{n}x{n}_nt{n_t}")
