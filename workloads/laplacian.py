"""Anisotropic 5-point Dirichlet Laplacian on an nx x ny grid, in CSR.

A = a_x (I_ny kron T_nx) + a_y (T_ny kron I_nx), T_m = tridiag(-1, 2, -1),
grid point (i, j) stored at row i + nx * j (x fastest).  Its eigenpairs are
known in closed form:
    lambda_{p,q} = a_x (2 - 2 cos(p pi/(nx+1))) + a_y (2 - 2 cos(q pi/(ny+1)))
    v_{p,q}(i, j) = sin(p pi (i+1)/(nx+1)) sin(q pi (j+1)/(ny+1))
for p = 1..nx, q = 1..ny.  Every diagonal entry is the same constant, so these
sine vectors are eigenvectors of the stored FP64 matrix as well.

This module builds inputs only; it holds no arithmetic of the refinement.
"""
import numpy as np


class Laplacian2D:
    def __init__(self, nx, ny, ax=1.0, ay=np.sqrt(2.0)):
        self.nx, self.ny, self.ax, self.ay = nx, ny, float(ax), float(ay)
        self.n = nx * ny

    def csr(self):
        """(row_ptr int32[n+1], col_idx int32[nnz], val float64[nnz]), columns sorted."""
        nx, ny, ax, ay = self.nx, self.ny, self.ax, self.ay
        n = self.n
        p = np.arange(n, dtype=np.int64)
        i, j = p % nx, p // nx
        # neighbour offsets in ascending column order
        offs = [(-nx, j > 0, -ay), (-1, i > 0, -ax), (0, np.ones(n, bool), 2 * ax + 2 * ay),
                (1, i < nx - 1, -ax), (nx, j < ny - 1, -ay)]
        cnt = sum(m.astype(np.int64) for _, m, _ in offs)
        row_ptr = np.zeros(n + 1, dtype=np.int64)
        np.cumsum(cnt, out=row_ptr[1:])
        nnz = int(row_ptr[-1])
        col = np.empty(nnz, dtype=np.int32)
        val = np.empty(nnz, dtype=np.float64)
        pos = row_ptr[:-1].copy()
        for off, mask, v in offs:
            rows = p[mask]
            col[pos[mask]] = (rows + off).astype(np.int32)
            val[pos[mask]] = v
            pos[mask] += 1
        return row_ptr.astype(np.int32), col, val

    def norm_inf(self):
        return 4.0 * self.ax + 4.0 * self.ay

    def eigenvalue(self, pq):
        p, q = pq
        return (self.ax * (2 - 2 * np.cos(p * np.pi / (self.nx + 1)))
                + self.ay * (2 - 2 * np.cos(q * np.pi / (self.ny + 1))))

    def smallest(self, count):
        """The ``count`` smallest (p, q) index pairs, ascending eigenvalue."""
        lim = int(np.ceil(np.sqrt(count))) + 4
        cands = [(p, q) for p in range(1, min(self.nx, 4 * lim) + 1)
                 for q in range(1, min(self.ny, 4 * lim) + 1)]
        cands.sort(key=self.eigenvalue)
        return cands[:count]

    def eigenvector(self, pq):
        p, q = pq
        sx = np.sin(p * np.pi * np.arange(1, self.nx + 1) / (self.nx + 1))
        sy = np.sin(q * np.pi * np.arange(1, self.ny + 1) / (self.ny + 1))
        v = np.outer(sy, sx).reshape(-1)        # index i + nx*j
        return v / np.linalg.norm(v)
