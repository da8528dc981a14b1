"""Pins of the oracle's variants beyond the plain sweep: Rayleigh--Ritz
preprocessing (Section 3.3), convergence judged on the leading k of K
columns (Section 4.1) and the shifted square B = A^2 - alpha I for the
smallest |eigenvalues| (Section 5.2).  Each is checked against what the
mathematics fixes, not against itself."""
import numpy as np

from oracle import refine as R
from workloads import configs as C


def random_orthogonal(k, seed):
    q, r = np.linalg.qr(np.random.default_rng(seed).standard_normal((k, k)))
    return q * np.sign(np.diag(r))[None, :]


def spread_problem(n=120, k=6, seed=11):
    # targets of distinct magnitude, the rest below them (|lambda| <= 0.7)
    lam = np.concatenate([np.array([1.0, -0.95, 0.9, -0.85, 0.8, -0.75])[:k], np.linspace(-0.7, 0.7, n - k)])
    return C.householder(n, 8, k, lam, seed, target="largest_mag", x_noise=0.0)


def test_rayleigh_ritz_invariants():
    p = spread_problem()
    X = p.X0 + 1e-3 * np.random.default_rng(1).standard_normal(p.X0.shape)
    Z, d = R.rayleigh_ritz(R.dense_operator(p.A), X)
    k = p.k
    assert np.abs(Z.T @ Z - np.eye(k)).max() < 1e-13
    D = Z.T @ p.A @ Z
    assert np.abs(D - np.diag(np.diag(D))).max() < 1e-13
    assert np.allclose(np.diag(D), d, atol=1e-13)
    assert np.all(np.diff(np.abs(d)) <= 0)                       # |d| descending


def test_rayleigh_ritz_recovers_a_rotated_and_scaled_eigenbasis():
    """X = Q_k M with M any nonsingular k x k (rotation and column scaling):
    the Ritz vectors are exactly the eigenvectors (up to sign), which needs the
    generalized problem -- M^T M != I."""
    p = spread_problem()
    M = random_orthogonal(p.k, 3) @ np.diag(np.linspace(0.5, 2.0, p.k))
    Z, d = R.rayleigh_ritz(R.dense_operator(p.A), p.Xtrue @ M)
    order = np.argsort(-np.abs(p.lam), kind="stable")
    Q = p.Xtrue[:, order]
    c = np.abs(np.einsum("ij,ij->j", Z, Q))
    assert np.all(c > 1 - 1e-13)
    assert np.allclose(d, p.lam[order], atol=1e-13)


def test_judged_columns_use_only_the_leading_block():
    p = spread_problem(k=6)
    X0 = p.X0.copy()
    X0[:, 3:] += 1e-3 * np.random.default_rng(2).standard_normal((p.n, 3))   # trailing columns far noisier
    X0 = C.orthonormalise(X0)
    op = R.dense_operator(p.A)
    _, full = R.refine(op, X0, p.normA, max_iters=3)
    _, same = R.refine(op, X0, p.normA, max_iters=3, judge_cols=6)
    _, lead = R.refine(op, X0, p.normA, max_iters=3, judge_cols=3)
    assert np.array_equal(full["hist_corr"], same["hist_corr"])
    # the first sweep's E, from the sign-fixed X0, restricted to three columns
    sigma = R.sign_fix(X0)
    _, info = R.refine_step(op, X0 * sigma[None, :], R.delta_threshold(p.normA))
    assert np.isclose(lead["hist_corr"][0], np.linalg.norm(info.E[:, :3]), rtol=1e-14)
    assert np.isclose(full["hist_corr"][0], np.linalg.norm(info.E), rtol=1e-14)
    assert lead["hist_corr"][0] < 0.1 * full["hist_corr"][0]


def test_shifted_square_has_the_squared_spectrum():
    lam = np.linspace(-1.0, 1.0, 90)
    p = C.householder(90, 8, 4, lam, 21, target="smallest_mag", x_noise=0.0)
    alpha = p.shift
    B = R.square_operator(p.A, alpha)
    Qall = p.gen.eigenvectors(np.arange(90))
    resid = B(Qall) - Qall * (lam * lam - alpha)[None, :]
    assert np.abs(resid).max() < 1e-13
    # the separation condition of Section 5.2 holds for this alpha
    order = np.argsort(np.abs(lam), kind="stable")
    tgt, rest = lam[order[:4]], lam[order[4:]]
    assert np.max(np.abs(rest ** 2 - alpha)) < np.min(np.abs(tgt ** 2 - alpha))


def test_shifted_square_refines_the_smallest_magnitudes():
    n, k = 150, 3
    # targets 0.1, -0.2, 0.3; the rest |lambda| in [0.5, 1] with alternating signs
    rest = np.linspace(0.5, 1.0, n - k) * np.where(np.arange(n - k) % 2 == 0, 1.0, -1.0)
    lam = np.concatenate([[0.1, -0.2, 0.3], rest])
    p = C.householder(n, 8, k, lam, 31, target="smallest_mag", x_noise=1e-6)
    norm_b = p.normA ** 2 + abs(p.shift)
    X, rep = R.refine(R.square_operator(p.A, p.shift), p.X0, p.normA, p.shift, max_iters=400,
                      tol=1e-14, norm_b=norm_b)
    assert rep["status"] == R.OK
    Xn = X / np.linalg.norm(X, axis=0)
    c = np.abs(np.einsum("ij,ij->j", Xn, p.Xtrue))
    assert np.all(1 - c < 1e-12)


def test_reorthonormalise_reaches_the_polar_factor():
    """Two Loewdin steps from ||X^T X - I|| ~ 1e-6 land on the closest matrix
    with orthonormal columns, the polar factor U V^T of X's SVD."""
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((200, 7)))
    X = Q + 1e-7 * rng.standard_normal(Q.shape)
    U, _, Vt = np.linalg.svd(X, full_matrices=False)
    Xr = R.reorthonormalise(X)
    assert np.abs(Xr.T @ Xr - np.eye(7)).max() < 2e-15
    assert np.abs(Xr - U @ Vt).max() < 1e-14


def axis_problem(n=60, k=3, seed=41):
    """A = diag(lambda) (no reflectors): the eigenvectors are unit vectors.
    X0 keeps column 0 exactly e_0 and perturbs the others below the leading
    block, so Y_1 = X_1 - I has a zero column unless the signs flip it."""
    lam = np.concatenate([[1.0, 0.9, 0.8], np.linspace(-0.5, 0.5, n - 3)])
    p = C.householder(n, 0, k, lam, seed, target="largest_mag", x_noise=0.0)
    X0 = p.Xtrue.copy()
    X0[k:, 1:] += 1e-6 * np.random.default_rng(seed).standard_normal((n - k, k - 1))
    return p, C.orthonormalise(X0)


def test_singular_leading_block_needs_the_signs():
    p, X0 = axis_problem()
    assert np.array_equal(X0[:, 0], p.Xtrue[:, 0])        # Y_1(:, 0) = 0 without the sign flip
    op = R.dense_operator(p.A)
    try:
        R.refine(op, X0, p.normA, max_iters=3, use_sign_fix=False)
        raised = False
    except R.SingularWY:
        raised = True
    assert raised
    X, rep = R.refine(op, X0, p.normA, max_iters=120, tol=1e-14, use_sign_fix=False, resign=True)
    assert rep["status"] == R.OK and rep["resigned"] == 1
    assert np.array_equal(rep["sigma"], [-1.0, -1.0, -1.0])
    c = np.abs(np.einsum("ij,ij->j", X / np.linalg.norm(X, axis=0), p.Xtrue))
    assert np.all(1 - c < 1e-14)
