"""Small problems with independently known eigenvectors, for the oracle pins.

A = Q diag(lam) Q^T with Q from Gram--Schmidt of a seeded Gaussian matrix; the
reference eigenvectors are recomputed from the stored FP64 matrix by the
oracle's Jacobi solver (not taken from the construction)."""
import numpy as np

from oracle.jacobi import jacobi_eigh
from workloads import rng
from workloads.dense import orthonormalise


class Small:
    def __init__(self, lam, seed, targets):
        lam = np.asarray(lam, dtype=np.float64)
        n = len(lam)
        Q = orthonormalise(rng.normal(seed, 0, n * n).reshape(n, n, order="F"))
        A = (Q * lam[None, :]) @ Q.T
        A = 0.5 * (A + A.T)
        w, V = jacobi_eigh(A)
        # match each requested eigenvalue to its Jacobi eigenpair
        order = [int(np.argmin(np.abs(w - lam[t]))) for t in targets]
        self.A, self.n, self.k = A, n, len(targets)
        self.w, self.V = w, V
        self.Vt = V[:, order]
        self.lam_t = w[order]
        rest = np.delete(np.arange(n), order)
        self.rest = rest
        self.normA = float(np.max(np.abs(w)))

    def perturbed(self, eps, seed, within=False):
        """V_T + eps * (random combination of the other eigenvectors)."""
        k = self.k
        if within:
            C = rng.normal(seed, 1, k * k).reshape(k, k)
            return self.Vt + eps * self.Vt @ C
        C = rng.normal(seed, 1, len(self.rest) * k).reshape(len(self.rest), k)
        return self.Vt + eps * self.V[:, self.rest] @ C


def separated(seed=11, n=40):
    """Targets 1.0, -0.95, 0.9; one eigenvalue -0.6 and the others on
    [-0.3, 0.3]: gamma = 2/3, next ratio 1/3."""
    lam = np.concatenate([[1.0, -0.95, 0.9, -0.6], np.linspace(-0.3, 0.3, n - 4)])
    return Small(lam, seed, targets=[0, 1, 2])


def delta_tie(gap_units, k=4, n=12, t=2.0 ** -10, seed=5):
    """An operator and an iterate whose Rayleigh quotients are exact binary64
    numbers: X = [0; I_k; 0] (columns e_k .. e_{2k-1}, exactly orthonormal),
    B symmetric with B[k+j, k+j] = d_j, d = (1, 1 + gap_units 2^-52, 0.6, 0.3),
    x_0^T B x_1 = t (so V_01 = x_0^T r_1 = t) and random couplings between
    the target rows and the others (a nonzero residual).  W = B X and the
    Rayleigh quotients are exact, so d_1 - d_0 = gap_units 2^-52; with ||B|| taken as
    2, delta = 10 * 2 * 2^-53 = 10 * 2^-52 (Section 3.1.3, choice of delta).
    Returns (B, X, norm_b)."""
    d = [1.0, 1.0 + gap_units * 2.0 ** -52, 0.6, 0.3]
    B = np.zeros((n, n))
    for j in range(k):
        B[k + j, k + j] = d[j]
    B[k, k + 1] = B[k + 1, k] = t
    others = list(range(k)) + list(range(2 * k, n))
    c = rng.uniform(seed, 0, len(others) * k).reshape(len(others), k) - 0.5
    for a, i in enumerate(others):
        B[i, i] = 0.05 * (a + 1)
        for j in range(k):
            # a few significant bits
            B[i, k + j] = B[k + j, i] = np.round(c[a, j] * 2 ** 8) * 2.0 ** -14
    X = np.zeros((n, k), order="F")
    X[np.arange(k, 2 * k), np.arange(k)] = 1.0
    return B, X, 2.0
