"""The block substitution behind the dense-block separator solves, restated in NumPy.

For a block-tridiagonal SPD matrix (the separators' Schur complement) with Cholesky factor L
(diagonal blocks D_K, sub-diagonal blocks E_K), the library solves L L^T x = r as
    z_K = D_K^{-1} r_K,  y_0 = z_0,  y_K = z_K - M_K y_{K-1},    M_K = D_K^{-1} E_K,
    w_K = D_K^{-T} y_K,  x_last = w_last,  x_K = w_K - P_K^T x_{K+1},  P_K = E_{K+1} D_K^{-1}.
This checks the identities against a direct solve (they are exact algebra; only rounding
differs), for one, two and several blocks.
"""
import numpy as np
import pytest


def block_tridiagonal_spd(nb, B, rng):
    n = nb * B
    A = np.zeros((n, n))
    for K in range(nb):
        G = rng.standard_normal((B, B))
        A[K * B:(K + 1) * B, K * B:(K + 1) * B] = G @ G.T + 4 * B * np.eye(B)
        if K + 1 < nb:
            E = rng.standard_normal((B, B))
            A[(K + 1) * B:(K + 2) * B, K * B:(K + 1) * B] = E
            A[K * B:(K + 1) * B, (K + 1) * B:(K + 2) * B] = E.T
    return A


@pytest.mark.parametrize("nb,B", [(1, 7), (2, 5), (6, 9)])
def test_block_substitution_with_inverted_diagonal_blocks(nb, B):
    rng = np.random.default_rng(nb * 100 + B)
    A = block_tridiagonal_spd(nb, B, rng)
    L = np.linalg.cholesky(A)
    blk = lambda M, K, J: M[K * B:(K + 1) * B, J * B:(J + 1) * B]  # noqa: E731
    # the factor is block bidiagonal (no fill left of the sub-diagonal block)
    for K in range(2, nb):
        assert np.all(L[K * B:(K + 1) * B, :(K - 1) * B] == 0.0)
    Dinv = [np.linalg.inv(blk(L, K, K)) for K in range(nb)]
    M = [Dinv[K] @ blk(L, K, K - 1) for K in range(1, nb)]        # M_K at K - 1
    P = [blk(L, K + 1, K) @ Dinv[K] for K in range(nb - 1)]        # P_K at K
    r = rng.standard_normal((nb * B, 3))
    rK = [r[K * B:(K + 1) * B] for K in range(nb)]
    y = [Dinv[K] @ rK[K] for K in range(nb)]
    for K in range(1, nb):
        y[K] = y[K] - M[K - 1] @ y[K - 1]
    x = [Dinv[K].T @ y[K] for K in range(nb)]
    for K in range(nb - 2, -1, -1):
        x[K] = x[K] - P[K].T @ x[K + 1]
    ref = np.linalg.solve(A, r)
    assert np.abs(np.concatenate(x) - ref).max() <= 1e-12 * np.abs(ref).max()
