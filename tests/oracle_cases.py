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
