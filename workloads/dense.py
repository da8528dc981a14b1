"""Dense symmetric test matrices A = Q diag(lam) Q^T with known eigenvectors.

Q = H_1 H_2 ... H_m is a product of m Householder reflectors
H_i = I - 2 v_i v_i^T / (v_i^T v_i) with seeded N(0,1) vectors v_i.  The
eigenpairs of A are (lam_i, Q e_i).  A is formed in FP64 through the
accumulated form Q = I - V C V^T (V holds the unit reflector vectors, C is
m x m upper triangular), which costs O(n^2 m) instead of O(n^3), and is made
exactly symmetric by construction (A = diag(lam) + Z + Z^T).

This module builds inputs only; it holds no arithmetic of the refinement.
"""
import numpy as np

from . import rng


def reflector_vectors(n, m, seed):
    """n x m matrix whose columns are the unit reflector vectors v_i / |v_i|."""
    V = rng.normal(seed, 1, n * m).reshape(m, n).T.copy()
    V /= np.linalg.norm(V, axis=0)
    return V


def accumulate(V):
    """C (m x m upper triangular) with H_1 ... H_m = I - V C V^T.

    Recurrence: appending H_j = I - 2 v v^T to I - V' C' V'^T gives the new
    last column [-2 C' (V'^T v); 2].
    """
    m = V.shape[1]
    C = np.zeros((m, m))
    for j in range(m):
        if j:
            C[:j, j] = -2.0 * C[:j, :j] @ (V[:, :j].T @ V[:, j])
        C[j, j] = 2.0
    return C


class HouseholderProblem:
    """A = Q diag(lam) Q^T with Q a product of ``m`` seeded reflectors."""

    def __init__(self, n, m, lam, seed):
        lam = np.asarray(lam, dtype=np.float64)
        assert lam.shape == (n,)
        self.n, self.m, self.lam, self.seed = n, m, lam, seed
        self.V = reflector_vectors(n, m, seed)
        self.C = accumulate(self.V)
        self.U = self.V @ self.C          # Q = I - U V^T

    def matrix(self, order="C"):
        """The n x n FP64 matrix A (exactly symmetric)."""
        U, V, lam = self.U, self.V, self.lam
        L = lam[:, None] * V                      # diag(lam) V
        K = V.T @ L                               # V^T diag(lam) V
        # A = diag(lam) - U L^T - L U^T + U K U^T = diag(lam) + Z + Z^T
        Z = U @ (0.5 * (K @ U.T) - L.T)
        A = Z + Z.T
        A[np.diag_indices(self.n)] += lam
        return np.ascontiguousarray(A) if order == "C" else np.asfortranarray(A)

    def eigenvectors(self, idx):
        """Columns Q e_i for the indices ``idx`` (n x len(idx), unit norm)."""
        idx = np.asarray(idx)
        Qc = -self.U @ self.V[idx, :].T
        Qc[idx, np.arange(len(idx))] += 1.0
        return Qc

    def apply(self, B):
        """Q @ B."""
        return B - self.U @ (self.V.T @ B)


def orthonormalise(X):
    """Classical Gram--Schmidt applied twice per column, in FP64."""
    X = np.array(X, dtype=np.float64, order="F", copy=True)
    k = X.shape[1]
    for j in range(k):
        x = X[:, j]
        for _ in range(2):
            if j:
                Qp = X[:, :j]
                x -= Qp @ (Qp.T @ x)
        x /= np.linalg.norm(x)
        X[:, j] = x
    return X


def fp32_round(X):
    return np.asarray(X, dtype=np.float32).astype(np.float64)
