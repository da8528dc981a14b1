"""ORACLE (test infrastructure only): the cyclic Jacobi method for the full
eigen-decomposition of a small real symmetric matrix (Golub & Van Loan,
Matrix Computations, Section 8.5), written out in plain numpy.  It is the
independent reference for eigenvectors of arbitrary symmetric matrices with
n <= 64 in the oracle's tests.
"""
import numpy as np


def jacobi_eigh(A, max_sweeps=60):
    """Eigenvalues (ascending) and orthonormal eigenvectors of symmetric A."""
    a = np.array(A, dtype=np.float64, copy=True)
    n = a.shape[0]
    v = np.eye(n)
    scale = np.linalg.norm(a)
    u = 2.0 ** -53
    for _ in range(max_sweeps):
        rotated = False
        for p in range(n - 1):
            for q in range(p + 1, n):
                apq = a[p, q]
                # negligible: below roundoff relative to the diagonal pair
                # (Demmel & Veselic's criterion) or to the whole matrix
                if abs(apq) <= u * np.sqrt(abs(a[p, p] * a[q, q])) or abs(apq) <= 1e-3 * u * scale / n:
                    continue
                rotated = True
                theta = (a[q, q] - a[p, p]) / (2.0 * apq)
                t = (1.0 if theta >= 0 else -1.0) / (abs(theta) + np.sqrt(theta * theta + 1.0))
                c = 1.0 / np.sqrt(t * t + 1.0)
                s = t * c
                tau = s / (1.0 + c)
                # Rutishauser's form of A <- J^T A J: the diagonal pair moves by
                # -/+ t a_pq, the other entries of rows/columns p, q rotate
                h = t * apq
                a[p, p] -= h
                a[q, q] += h
                a[p, q] = a[q, p] = 0.0
                r = np.r_[0:p, p + 1:q, q + 1:n]
                g, hq = a[r, p].copy(), a[r, q].copy()
                a[r, p] = g - s * (hq + g * tau)
                a[r, q] = hq + s * (g - hq * tau)
                a[p, r] = a[r, p]
                a[q, r] = a[r, q]
                vp, vq = v[:, p].copy(), v[:, q].copy()
                v[:, p] = vp - s * (vq + vp * tau)
                v[:, q] = vq + s * (vp - vq * tau)
        if not rotated:
            break
    w = np.diag(a).copy()
    order = np.argsort(w)
    return w[order], v[:, order]
