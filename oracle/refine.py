"""ORACLE (test infrastructure only): the refinement method, step by step, in
plain numpy FP64, in the paper's literal form (explicit Y-hat, T-hat, V and
E-tilde_L; the orthogonal H-hat is applied through its compact WY factors and
never formed).

Paper: Terao, Ozaki, Imamura, Ogita, "Iterative Refinement for a Subset of
Eigenvectors of Symmetric Matrices via Matrix Multiplications".
Readings of points the paper leaves open are marked READING and listed with
their reasons in the design notes.
"""
import numpy as np

U_FP64 = 2.0 ** -53          # unit roundoff of binary64 (Section 3.1.3, choice of delta)


class SingularWY(np.linalg.LinAlgError):
    """Algorithm 1 needs a nonsingular leading block Y_1 (Section 3.1.1)."""


def compact_wy(Q):
    """Algorithm 1, CompactWY(Q): Y = Q - I_{n,k}, T = -Y_1^{-T}.

    Ensures (for Q with orthonormal columns) Q = (I - Y T Y^T) I_{n,k} and that
    I - Y T Y^T is orthogonal.  T is obtained by an LU solve with partial
    pivoting, not an explicit inverse.
    """
    n, k = Q.shape
    Y = np.array(Q, dtype=np.float64, copy=True)
    Y[np.arange(k), np.arange(k)] -= 1.0
    Y1 = Y[:k, :k]
    if not np.all(np.isfinite(Y1)) or np.linalg.cond(Y1) > 1.0 / (k * U_FP64):
        raise SingularWY("leading k x k block of Y is singular to working precision")
    T = -np.linalg.solve(Y1.T, np.eye(k))     # Y_1^T (-T) = I
    return Y, T


def sign_of(v):
    """READING: sign(0) := +1 in Algorithm 2 (the paper leaves sign(0) open;
    MATLAB's sign(0) = 0 would make the pivot q_jj - sigma_j zero)."""
    return 1.0 if v >= 0 else -1.0


def modified_lu(Q):
    """Algorithm 2, modified_LU(Q): unpivoted LU of Q - Sigma with
    sigma_j = -sign(q_jj) chosen at step j.  Returns (Y, U, sigma) with
    Y unit lower trapezoidal (n x k), U upper triangular (k x k) and
    Q - [diag(sigma); 0] = Y U."""
    q = np.array(Q, dtype=np.float64, copy=True)
    n, k = q.shape
    sigma = np.empty(k)
    for j in range(k):
        sigma[j] = -sign_of(q[j, j])
        q[j, j] -= sigma[j]
        q[j + 1:, j] /= q[j, j]
        q[j + 1:, j + 1:k] -= np.outer(q[j + 1:, j], q[j, j + 1:k])
    U = np.triu(q[:k, :k])
    Y = np.tril(q, -1)
    Y[np.arange(k), np.arange(k)] = 1.0
    return Y, U, sigma


def compact_wy_lu(Q):
    """Algorithm 3, CompactWY_LU(Q): [Y, U, Sigma] = modified_LU(Q),
    T = -U Sigma Y_1^{-T}.

    READING: with this T the WY matrix satisfies (I - Y T Y^T) I_{n,k} = Q Sigma
    (the columns of Q with the signs sigma), which equals Q only when Sigma = I;
    the orthogonality of I - Y T Y^T holds as stated.
    """
    Y, U, sigma = modified_lu(Q)
    k = Q.shape[1]
    Y1 = Y[:k, :k]
    T = -(U * sigma[None, :]) @ np.linalg.solve(Y1.T, np.eye(k))   # -U Sigma Y_1^{-T}
    return Y, T, sigma


def sign_fix(X):
    """The practical rule closing Section 3.1.1: the signs sigma of
    Algorithm 2, applied once as X <- X Sigma, make Algorithm 1 applicable.

    sigma depends only on the leading k x k block (the pivots of Algorithm 2
    never read rows > k), so it is computed from that block alone.
    READING: applied always, at the start of every refinement call, and undone
    on exit.
    """
    k = X.shape[1]
    _, _, sigma = modified_lu(X[:k, :k])
    return sigma


def apply_h(Y, T, B):
    """H-hat B = B - Y (T (Y^T B)) (compact WY application, Section 3.1.2)."""
    return B - Y @ (T @ (Y.T @ B))


def apply_ht(Y, T, B):
    """H-hat^T B = B - Y (T^T (Y^T B))."""
    return B - Y @ (T.T @ (Y.T @ B))


class StepInfo(dict):
    __getattr__ = dict.__getitem__


def refine_step(apply_b, Xh, delta, beta="cluster"):
    """Algorithm 4: one refinement step X-tilde = X-hat + H-hat E-tilde_L.

    apply_b(X) returns B X for the operator whose dominant eigenvectors are
    refined (B = A, or the shifted A - alpha I of Section 5).
    beta = "cluster": beta_ij = -x_i^T x_j / 2 (near-equal Rayleigh quotients),
    beta = "zero":    beta_ij = 0 (after a Rayleigh--Ritz preprocessing).
    """
    n, k = Xh.shape
    W = apply_b(Xh)                                     # W = A X-hat
    Y, T = compact_wy(Xh)                               # compact WY factors, Algorithm 1
    alpha = np.einsum("ij,ij->j", Xh, Xh)               # alpha_j = x_j^T x_j
    d = np.einsum("ij,ij->j", Xh, W) / alpha            # Rayleigh quotients, Eq. (Rayleigh)
    R = W - Xh * d[None, :]                             # W - X-hat D-tilde_1
    V = apply_ht(Y, T, R)                               # V = H-hat^T (W - X-hat D-tilde_1), Eq. (V-def)
    E = np.empty((n, k))
    for i in range(k):                                  # E-tilde_L by its four cases, Eqs. (Ediag), (Eoffdiag)
        for j in range(k):
            if i == j:
                E[i, j] = (1.0 - alpha[i]) / 2.0
            elif abs(d[j] - d[i]) <= delta:
                E[i, j] = -(Xh[:, i] @ Xh[:, j]) / 2.0 if beta == "cluster" else 0.0
            else:
                E[i, j] = V[i, j] / (d[j] - d[i])
    E[k:, :] = V[k:, :] / d[None, :]
    Xt = Xh + apply_h(Y, T, E)                          # X-hat + H-hat E-tilde_L, Eq. (update-X)
    return Xt, StepInfo(d=d, alpha=alpha, R=R, V=V, E=E, Y=Y, T=T, W=W,
                        res_fro=float(np.linalg.norm(R)), e_fro=float(np.linalg.norm(E)))


def reorthonormalise(X, steps=2):
    """The optional reorthogonalisation of Section 3.1.3.  READING: symmetric
    (Loewdin) steps X <- X (3 I - X^T X) / 2, the first-order expansion of
    X (X^T X)^{-1/2}; each step squares ||X^T X - I||."""
    k = X.shape[1]
    for _ in range(steps):
        X = X @ (1.5 * np.eye(k) - 0.5 * (X.T @ X))
    return X


def normalise(X):
    """Column normalisation after each update (Section 3.1.3, precision and
    orthogonality)."""
    return X / np.linalg.norm(X, axis=0)[None, :]


def delta_threshold(norm_b, c=10.0):
    """delta = c ||A|| u, c = 10 (Section 3.1.3, choice of delta).
    READING: ||.|| is the norm of the refined operator B = A - alpha I,
    bounded by ||A|| + |alpha|."""
    return c * norm_b * U_FP64


STOP_CORRECTION, STOP_RESIDUAL = 0, 1
OK, E_DIVERGED, E_NOT_CONVERGED, E_NONFINITE = 0, 5, 6, 7


def rayleigh_ritz(apply_b, X):
    """Rayleigh--Ritz preprocessing (Section 3.3, handling clustered
    eigenvalues): solve (X^T B X) S = (X^T X) S D and return Z = X S with
    Z^T Z = I and Z^T B Z = D.  The generalized symmetric eigensolver of scipy
    is the step for the k x k problem.  READING: the Ritz pairs are ordered by
    |D| descending (the refinement targets the largest |eigenvalues| of B), and
    each Ritz vector's sign makes its largest-magnitude entry positive.
    Returns (Z, d)."""
    import scipy.linalg as sla
    W = apply_b(X)
    G = X.T @ X
    Sm = X.T @ W
    Sm = 0.5 * (Sm + Sm.T)           # X^T B X is symmetric; drop its rounding asymmetry
    d, S = sla.eigh(Sm, G)
    order = np.argsort(-np.abs(d), kind="stable")
    d, S = d[order], S[:, order]
    Z = X @ S
    piv = np.argmax(np.abs(Z), axis=0)
    sg = np.where(Z[piv, np.arange(Z.shape[1])] < 0, -1.0, 1.0)
    return np.asfortranarray(Z * sg[None, :]), d


def refine(apply_b, X0, norm_a, shift=0.0, max_iters=10, tol=0.0, stop=STOP_CORRECTION,
           delta_c=10.0, beta="cluster", div_factor=10.0, div_floor=1e-4, use_sign_fix=True,
           rayleigh_ritz_first=False, judge_cols=0, norm_b=None, resign=False):
    """Iterate Algorithm 4 with the driver choices of Section 3.1.3.

    Per sweep t: R_t and E_t are computed from X_t, the update is applied and
    the columns normalised, giving X_{t+1}.  Stopping (READING): stop with
    X_{t+1} once ||E_t||_F <= tol (correction-size criterion) or
    ||R_t||_F / ||A|| <= tol (backward-error criterion); tol = 0 runs exactly
    max_iters sweeps.  Divergence (the advice closing Section 4.3.1;
    READING): stop once ||E_t||_F >= 1 (the Neumann-series assumption
    ||E|| < 1 of Section 3.1.2 fails) or ||E_t||_F exceeds div_factor times
    the smallest earlier value and div_floor.  A non-finite sweep leaves the
    last finite iterate.

    rayleigh_ritz_first: replace X0 by its Ritz vectors first (Section 3.3).
    judge_cols: with K = X0's column count > judge_cols > 0, the stop and
    divergence tests use the correction of the leading judge_cols columns only
    (Section 4.1: K vectors refined, convergence judged on the leading k).
    norm_b: ||B|| for delta and the residual test when B is not A - shift I
    (the shifted square of Section 5.2); default ||A|| + |shift| and ||A||.
    resign: when Algorithm 1 meets a singular Y_1 mid-run, take the signs of
    Algorithm 2 for the current X (the choice Algorithm 3 builds into its WY
    factors), X <- X Sigma, and redo the sweep (at most 4 times per call).

    Returns (X, report) with X in the caller's column signs (or, after the
    Rayleigh--Ritz step, in its order and signs).
    """
    X = np.array(X0, dtype=np.float64, order="F", copy=True)
    k = X.shape[1]
    if rayleigh_ritz_first:
        X, _ = rayleigh_ritz(apply_b, X)
    sigma = sign_fix(X) if use_sign_fix else np.ones(k)
    X = X * sigma[None, :]
    delta = delta_threshold(norm_a + abs(shift) if norm_b is None else norm_b, delta_c)
    res_scale = norm_a if norm_b is None else norm_b
    kj = judge_cols if 0 < judge_cols < k else k
    hist_r, hist_e = [], []
    status, it, d = E_NOT_CONVERGED if tol > 0 else OK, 0, None
    emin = np.inf
    resigned = 0
    for t in range(max_iters):
        while True:
            try:
                Xn, info = refine_step(apply_b, X, delta, beta)
                break
            except SingularWY:
                if not resign or resigned >= 4:
                    raise
                s2 = sign_fix(X)
                X = X * s2[None, :]
                sigma = sigma * s2
                resigned += 1
        rel_r = info.res_fro / res_scale
        e_fro = info.e_fro if kj == k else float(np.linalg.norm(info.E[:, :kj]))
        if not (np.all(np.isfinite(Xn)) and np.isfinite(e_fro) and np.isfinite(rel_r)):
            status = E_NONFINITE
            break
        hist_r.append(rel_r)
        hist_e.append(e_fro)
        d = info.d
        X = normalise(Xn)
        it += 1
        crit = e_fro if stop == STOP_CORRECTION else rel_r
        if tol > 0 and crit <= tol:
            status = OK
            break
        if e_fro >= 1.0 or (e_fro > div_factor * emin and e_fro > div_floor):
            status = E_DIVERGED
            break
        emin = min(emin, e_fro)
    X = X * sigma[None, :]
    return X, dict(status=status, iterations=it, d=None if d is None else d + shift,
                   hist_res=np.array(hist_r), hist_corr=np.array(hist_e), sigma=sigma,
                   delta=delta, resigned=resigned)


def dense_operator(A, shift=0.0):
    """B X = A X - shift X for a dense FP64 matrix."""
    A = np.asarray(A)
    return lambda X: A @ X - shift * X


def square_operator(A, alpha):
    """B X = A (A X) - alpha X: the shifted square of Section 5.2 (smallest
    |eigenvalues|), A^2 never formed."""
    A = np.asarray(A)
    return lambda X: A @ (A @ X) - alpha * X


def csr_operator(row_ptr, col_idx, val, n, shift=0.0):
    """B X = A X - shift X for a CSR matrix (scipy's sparse product as the step)."""
    import scipy.sparse as sp
    A = sp.csr_matrix((val, col_idx, row_ptr), shape=(n, n))
    return lambda X: A @ X - shift * X


def csr_square_operator(row_ptr, col_idx, val, n, alpha):
    """B X = A (A X) - alpha X for a CSR matrix."""
    import scipy.sparse as sp
    A = sp.csr_matrix((val, col_idx, row_ptr), shape=(n, n))
    return lambda X: A @ (A @ X) - alpha * X
