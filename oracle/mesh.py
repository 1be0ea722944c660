"""Structured triangular mesh of the rectangle [0, Lx] x [0, Ly].

The paper's experiments (Sec. 4, "uniform right triangular grid", refinement by
joining edge midpoints) use a uniform grid of right triangles with spacing
h = 1/2^k. Reading (diagonal direction, unspecified in the paper): each square
cell (i, j) is split along its "/" diagonal into the lower triangle
(i,j)-(i+1,j)-(i+1,j+1) and the upper triangle (i,j)-(i+1,j+1)-(i,j+1), both
counter-clockwise. Node (i, j) has index j (n+1) + i. Triangle 2 (j n + i) is the
lower and 2 (j n + i) + 1 the upper triangle of cell (i, j).
"""
import numpy as np


def structured_mesh(n: int, Lx: float = 1.0, Ly: float = 1.0):
    """Return (coords [(n+1)^2, 2] float64, tris [2 n^2, 3] int64)."""
    nx = n + 1
    coords = np.zeros((nx * nx, 2))
    for j in range(nx):
        for i in range(nx):
            coords[j * nx + i] = (i * (Lx / n), j * (Ly / n))
    tris = np.zeros((2 * n * n, 3), dtype=np.int64)
    for j in range(n):
        for i in range(n):
            v00 = j * nx + i
            v10 = v00 + 1
            v01 = v00 + nx
            v11 = v01 + 1
            e = 2 * (j * n + i)
            tris[e] = (v00, v10, v11)
            tris[e + 1] = (v00, v11, v01)
    return coords, tris


def boundary_nodes(n: int):
    """Dict of node-index arrays for the four sides: 'bottom' (y=0), 'top' (y=Ly),
    'left' (x=0), 'right' (x=Lx). Corners belong to two sides."""
    nx = n + 1
    idx = np.arange(nx)
    return {
        "bottom": idx,
        "top": n * nx + idx,
        "left": idx * nx,
        "right": idx * nx + n,
    }
