"""Pins of one refinement step (Algorithm 4) and of the driver against what the
paper's analysis fixes: the fixed point, the first-order decay law of the
non-target components (ratio lambda_i / lambda_j, Section 3.2), the quadratic
contraction of target-target components (Lemma 3.2), the diagonal and
clustered (beta) branches, the linear rate gamma, and the attainable accuracy
(Section 4.2)."""
import numpy as np
import pytest

from oracle import dd, refine as R
from tests.oracle_cases import Small, separated


def step(case, X, delta_c=10.0, beta="cluster"):
    delta = R.delta_threshold(case.normA, delta_c)
    return R.refine_step(R.dense_operator(case.A), X, delta, beta)


def coeffs(case, X):
    """c_ij = v_i^T x_j in the Jacobi eigenbasis."""
    return case.V.T @ X


def test_fixed_point():
    c = separated()
    Xn, info = step(c, c.Vt.copy())
    # the Jacobi reference itself is orthonormal only to ~1e-14
    assert np.abs(Xn - c.Vt).max() < 1e-13
    assert np.abs(info.E).max() < 1e-13
    assert np.abs(info.d - c.lam_t).max() < 1e-13


def test_first_order_decay_law():
    """Non-target component i of column j is multiplied by lambda_i / lambda_j."""
    c = separated()
    eps = 1e-6
    X = c.perturbed(eps, seed=3)
    before = coeffs(c, X)
    Xn, _ = step(c, X)
    after = coeffs(c, Xn)
    for jj in range(c.k):
        ratio = c.w[c.rest] / c.lam_t[jj]
        pred = ratio * before[c.rest, jj]
        # deviation is second order in eps (first-order mistakes leave ~eps)
        assert np.abs(after[c.rest, jj] - pred).max() < 50 * eps ** 2


def test_target_block_contracts_quadratically():
    c = separated()
    eps = 1e-6
    X = c.perturbed(eps, seed=4, within=True)
    Xn, info = step(c, X)
    C = coeffs(c, Xn)
    tgt = [int(np.argmin(np.abs(c.w - l))) for l in c.lam_t]
    off = C[tgt, :] - np.diag(np.diag(C[tgt, :]))
    assert np.abs(off).max() < 50 * eps ** 2
    assert np.abs(info.d - c.lam_t).max() < 50 * eps ** 2


def test_diagonal_branch_normalises():
    """e_jj = (1 - x_j^T x_j)/2 restores unit norm to second order."""
    c = separated()
    eta = 1e-6
    X = c.Vt * (1.0 + eta * np.array([1.0, -2.0, 3.0]))[None, :]
    Xn, _ = step(c, X)
    assert np.abs(np.linalg.norm(Xn, axis=0) - 1.0).max() < 50 * eta ** 2


def test_cluster_branch_restores_orthogonality():
    """With every pair treated as clustered, beta_ij = -x_i^T x_j / 2 removes
    the first-order loss of orthogonality."""
    c = separated()
    eps = 1e-6
    S = np.array([[0.0, 1.0, -2.0], [1.0, 0.0, 0.5], [-2.0, 0.5, 0.0]])
    X = c.Vt @ (np.eye(3) + eps * S)
    Xn, _ = step(c, X, delta_c=1e30)
    G = Xn.T @ Xn
    assert np.abs(G - np.eye(3)).max() < 50 * eps ** 2
    # beta = 0 (after preprocessing) leaves the first-order error in place
    Xz, _ = step(c, X, delta_c=1e30, beta="zero")
    assert np.abs(Xz.T @ Xz - np.eye(3)).max() > 0.5 * eps


def test_linear_rate_is_gamma():
    """Per-vector asymptotic factor max_{i>k}|lambda_{p_i}| / |lambda_{p_j}|
    (Section 3.2, the limit stated before Theorem 3.5); gamma is the slowest."""
    c = separated()
    gamma = np.max(np.abs(c.w[c.rest])) / np.min(np.abs(c.lam_t))
    assert abs(gamma - 2 / 3) < 1e-12
    X = c.perturbed(1e-3, seed=5)
    sines = []
    for _ in range(24):
        X, _ = step(c, X)
        X = R.normalise(X)
        sines.append(dd.sin_angles(X, c.Vt))
    sines = np.array(sines)
    rates = sines[16:24] / sines[15:23]
    pred = np.max(np.abs(c.w[c.rest])) / np.abs(c.lam_t)
    assert np.all(np.abs(rates - pred[None, :]) < 0.01), (rates, pred)
    # the Frobenius correction norm decays no faster than gamma
    _, rep = R.refine(R.dense_operator(c.A), c.perturbed(1e-3, seed=5), c.normA, max_iters=24)
    e = rep["hist_corr"]
    assert np.all(e[11:24] / e[10:23] < gamma + 0.005)


def test_converges_to_reference_eigenvectors():
    c = separated()
    X0 = c.perturbed(1e-4, seed=6)
    X, rep = R.refine(R.dense_operator(c.A), X0, c.normA, max_iters=200, tol=1e-15,
                      stop=R.STOP_RESIDUAL)
    assert rep["status"] == R.OK
    assert dd.sin_angles(X, c.Vt).max() < 1e-13
    assert np.abs(dd.orth_error(X)).max() < 1e-14
    _, res = dd.residual_dense(c.A, X)
    assert res.max() < 10 * R.U_FP64 * c.normA      # attainable residual O(u)||A||
    assert np.abs(rep["d"] - c.lam_t).max() < 1e-14


@pytest.mark.parametrize("which", ["smallest", "largest"])
def test_shift_variants(which):
    """Section 5.1: the k smallest (or largest) eigenvalues through B = A - alpha I."""
    lam = np.linspace(-1.0, 1.0, 36)
    tg = [0, 1, 2] if which == "smallest" else [35, 34, 33]
    c = Small(lam, seed=12, targets=tg)
    lam_kp1 = lam[3] if which == "smallest" else lam[32]
    alpha = (c.normA + lam_kp1) / 2 if which == "smallest" else (lam_kp1 - c.normA) / 2
    X0 = c.perturbed(1e-6, seed=7)
    X, rep = R.refine(R.dense_operator(c.A, alpha), X0, c.normA, shift=alpha, max_iters=3000,
                      tol=1e-15, stop=R.STOP_RESIDUAL)
    assert rep["status"] == R.OK
    assert dd.sin_angles(X, c.Vt).max() < 1e-12
    assert np.abs(rep["d"] - c.lam_t).max() < 1e-14


def test_stop_on_correction_size():
    c = separated()
    X0 = c.perturbed(1e-4, seed=8)
    _, full = R.refine(R.dense_operator(c.A), X0, c.normA, max_iters=40)
    tol = full["hist_corr"][9] * 1.0000001
    _, rep = R.refine(R.dense_operator(c.A), X0, c.normA, max_iters=40, tol=tol)
    assert rep["status"] == R.OK and rep["iterations"] == 10
    assert np.array_equal(rep["hist_corr"], full["hist_corr"][:10])


def test_not_converged_status():
    c = separated()
    _, rep = R.refine(R.dense_operator(c.A), c.perturbed(1e-3, seed=9), c.normA, max_iters=3, tol=1e-15)
    assert rep["status"] == R.E_NOT_CONVERGED and rep["iterations"] == 3


def test_nonfinite_keeps_last_finite_iterate():
    c = separated()
    X0 = c.perturbed(1e-4, seed=10)
    X0[5, 1] = np.nan
    X, rep = R.refine(R.dense_operator(c.A), X0, c.normA, max_iters=5)
    assert rep["status"] == R.E_NONFINITE and rep["iterations"] == 0


def test_sign_fix_is_undone():
    c = separated()
    X0 = c.perturbed(1e-5, seed=11) * np.array([1.0, -1.0, 1.0])[None, :]
    X, _ = R.refine(R.dense_operator(c.A), X0, c.normA, max_iters=5)
    assert np.all(np.sum(X * X0, axis=0) > 0.99)
