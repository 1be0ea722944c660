"""The bench's algorithmic flop count of the exact block solves, against the factors themselves.

bench.band_solve_flops counts 2 flop per structurally nonzero off-diagonal factor entry per
column and triangular solve: strip interiors by their factors' row envelopes (within the
half-band d (w + 2) - 1 the band kernels sweep; w the strip's width in nodes, d = 2 for A and 1
for S), the separators' Schur complement as a block-bidiagonal factor with d (n + 1) x d (n + 1)
blocks, plus the two sparse couplings. Here the oracle's
assembly pattern (every field pair of adjacent nodes, the pattern the library stores) is given
generic symmetric positive definite values, put into the same strip / separator ordering, the
Schur complement is formed and every factor is computed densely on a small mesh: the count is the
symbolic one (entries that the pattern does not force to zero), which Cholesky of generic values
fills exactly. The assembled values have a few more zeros than their pattern (on "/"-split right
triangles the Laplacian's diagonal-neighbour coupling vanishes, and the elimination drops the
Dirichlet DOFs' columns), so the useful work is somewhat below the count; that is checked too.
"""
import os
import sys

import numpy as np
import pytest

import workloads as W
from oracle import fem
from oracle.mesh import structured_mesh
from oracle.system import build_system

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
import bench  # noqa: E402


def layout(n, k):
    """strip widths and first node columns, separator node columns (k strips of n + 1 columns)"""
    C = n + 1
    ni = C - (k - 1)
    width = [ni // k + (1 if t < ni % k else 0) for t in range(k)]
    start, sep, x = [], [], 0
    for t in range(k):
        start.append(x)
        x += width[t]
        if t < k - 1:
            sep.append(x)
            x += 1
    return width, start, sep


def blocks(case, assembled=False):
    """A (u-block, index 2 v + f) and S (index v): the assembled blocks (after the Dirichlet
    elimination), or generic SPD matrices with their pattern (seeded values, diagonally dominant)"""
    s = build_system(case)
    u, p = s.u_idx, s.p_idx
    if assembled:
        AA = s.AA.tocsr()
        return {2: AA[u][:, u].toarray(), 1: (-AA[p][:, p]).toarray()}
    coords, tris = structured_mesh(case.n)
    rp, col = fem.csr_pattern(tris, 3 * coords.shape[0])
    nd = 3 * coords.shape[0]
    P = np.zeros((nd, nd))
    P[np.repeat(np.arange(nd), np.diff(rp)), col] = 1.0
    rng = np.random.default_rng(0)
    out = {}
    for d, idx in ((2, u), (1, p)):
        M = P[np.ix_(idx, idx)] * rng.uniform(0.5, 1.5, (len(idx), len(idx)))
        M = np.triu(M) + np.triu(M, 1).T
        out[d] = M + np.diag(np.abs(M).sum(axis=1) + 1.0)
    return out


def strip_index(n, d, cols):
    """natural block indices of the nodes in node columns `cols`, rows j outer, columns, fields"""
    C = n + 1
    return np.array([d * (j * C + i) + f for j in range(C) for i in cols for f in range(d)])


def strict_lower_nnz(L):
    return int(np.count_nonzero(np.tril(L, -1)))


@pytest.mark.parametrize("n,k", [(12, 3), (16, 2), (20, 4)])
def test_counted_structure_matches_the_factors(n, k):
    case = W.terzaghi_small().with_(n=n, n_t=2)
    mats = blocks(case)
    width, start, sep = layout(n, k)
    C = n + 1
    brute = 0.0
    for d in (2, 1):
        A = mats[d]
        interior_nnz, interior_count = 0, 0.0
        Ainv_IS = []
        sep_idx = np.concatenate([strip_index(n, d, [c]) for c in sep])
        for t in range(k):
            idx = strip_index(n, d, range(start[t], start[t] + width[t]))
            Att = A[np.ix_(idx, idx)]
            r, c = np.nonzero(Att)
            b = d * (width[t] + 2) - 1
            assert np.abs(r - c).max() == b, (d, t)  # the strip's half-band in this ordering
            L = np.linalg.cholesky(Att)
            assert np.all(np.tril(L, -b - 1) == 0.0)  # no fill outside the band
            interior_nnz += strict_lower_nnz(L)
            interior_count += bench.strip_envelope(width[t], C, d)
            Ainv_IS.append((idx, np.linalg.solve(Att, A[np.ix_(idx, sep_idx)])))
        assert interior_nnz == interior_count, (interior_nnz, interior_count)
        # separators' Schur complement, strip by strip (exact zeros between separators that
        # share no strip), and its factor: block bidiagonal, exact zeros left of block m - 1
        Ssep = A[np.ix_(sep_idx, sep_idx)].copy()
        for idx, Z in Ainv_IS:
            Ssep -= A[np.ix_(sep_idx, idx)] @ Z
        B, nb = d * C, k - 1
        Ls = np.linalg.cholesky(Ssep)
        for m in range(2, nb):
            assert np.all(Ls[m * B:(m + 1) * B, :(m - 1) * B] == 0.0)
        sep_nnz = strict_lower_nnz(Ls)
        sep_count = B * (B - 1) / 2.0 + (nb - 1) * (B * B + B * (B - 1) / 2.0)
        assert sep_nnz == sep_count, (sep_nnz, sep_count)
        # couplings: separator rows against interior columns
        interior_idx = np.concatenate([idx for idx, _ in Ainv_IS])
        cpl_nnz = np.count_nonzero(A[np.ix_(sep_idx, interior_idx)])
        cpl_count = (k - 1) * (4 * C - 2) * d * d
        assert cpl_nnz == cpl_count, (cpl_nnz, cpl_count)
        # one column: two forward + backward pairs on the interiors, one on the separators,
        # two couplings, 2 flop per entry
        brute += 2.0 * (4 * interior_nnz + 2 * sep_nnz + 2 * cpl_nnz)

    class Info:
        n_nodes = C * C
    counted, launches = bench.band_solve_flops(Info, 1, "diag", k, (True, True))
    assert brute == pytest.approx(counted, rel=1e-12), (brute, counted)
    assert launches == 2 * (8 + 2 * (k - 1))


def test_assembled_factors_need_no_more_than_the_count():
    # the assembled (eliminated) strip factors have at most the counted entries: their zeros
    # beyond the pattern's only lower the useful work
    n, k = 24, 3
    width, start, sep = layout(n, k)
    mats = blocks(W.terzaghi_small().with_(n=n, n_t=2), assembled=True)
    for d in (2, 1):
        for t in range(k):
            idx = strip_index(n, d, range(start[t], start[t] + width[t]))
            nnz = strict_lower_nnz(np.linalg.cholesky(mats[d][np.ix_(idx, idx)]))
            assert 0.7 * bench.strip_envelope(width[t], n + 1, d) < nnz <= bench.strip_envelope(width[t], n + 1, d)
