"""Pins of the oracle's compact-WY constructions (Algorithms 1-3) against the
properties the paper states for them, checked on explicitly formed matrices."""
import numpy as np
import pytest

from oracle import refine as R
from workloads import rng
from workloads.dense import orthonormalise


def rand_orth(n, k, seed):
    return orthonormalise(rng.normal(seed, 0, n * k).reshape(n, k, order="F"))


def explicit_h(Y, T):
    n = Y.shape[0]
    return np.eye(n) - Y @ T @ Y.T


@pytest.mark.parametrize("n,k,seed", [(40, 6, 1), (17, 16, 2), (64, 1, 3)])
def test_alg1_postcondition(n, k, seed):
    Q = rand_orth(n, k, seed)
    Y, T = R.compact_wy(Q)
    H = explicit_h(Y, T)
    assert np.abs(H[:, :k] - Q).max() < 1e-13           # Q = (I - Y T Y^T) I_{n,k}
    assert np.abs(H.T @ H - np.eye(n)).max() < 1e-13    # orthogonal
    # Y = Q - I_{n,k} exactly, T = -Y1^{-T}
    assert np.array_equal(Y[k:], Q[k:])
    assert np.abs(T.T @ Y[:k, :k] + np.eye(k)).max() < 1e-13


def test_wy_application_matches_explicit():
    Q = rand_orth(30, 5, 4)
    Y, T = R.compact_wy(Q)
    B = rng.normal(4, 9, 30 * 5).reshape(30, 5)
    H = explicit_h(Y, T)
    assert np.abs(R.apply_h(Y, T, B) - H @ B).max() < 1e-13
    assert np.abs(R.apply_ht(Y, T, B) - H.T @ B).max() < 1e-13


def singular_case():
    # q_11 = 1 exactly: Y_1 has a zero first row, Algorithm 1 cannot run
    Q = rand_orth(20, 4, 5)
    Q[:, 0] = 0.0
    Q[0, 0] = 1.0
    return orthonormalise(Q)


def test_alg1_fails_on_singular_leading_block():
    with pytest.raises(R.SingularWY):
        R.compact_wy(singular_case())


@pytest.mark.parametrize("seed", [6, 7])
def test_alg2_factorisation(seed):
    Q = rand_orth(25, 7, seed)
    Y, U, sigma = R.modified_lu(Q)
    S = np.zeros_like(Q)
    S[np.arange(7), np.arange(7)] = sigma
    assert np.abs(Q - S - Y @ U).max() < 1e-13          # Q - Sigma = Y U
    assert np.array_equal(np.triu(U), U)
    assert np.array_equal(np.diag(Y[:7]), np.ones(7))
    assert np.array_equal(np.triu(Y[:7], 1), np.zeros((7, 7)))
    assert set(np.unique(sigma)) <= {-1.0, 1.0}


@pytest.mark.parametrize("Q", [rand_orth(25, 7, 8), singular_case()])
def test_alg3_orthogonal_and_maps_to_signed_q(Q):
    n, k = Q.shape
    Y, T, sigma = R.compact_wy_lu(Q)
    H = explicit_h(Y, T)
    assert np.abs(H.T @ H - np.eye(n)).max() < 1e-13
    # (I - Y T Y^T) I_{n,k} = Q Sigma (the reading of Algorithm 3's postcondition)
    assert np.abs(H[:, :k] - Q * sigma[None, :]).max() < 1e-13


def test_sign_fix_rescues_alg1():
    Q = singular_case()
    sigma = R.sign_fix(Q)
    Y, T = R.compact_wy(Q * sigma[None, :])
    H = explicit_h(Y, T)
    assert np.abs(H[:, :4] - Q * sigma[None, :]).max() < 1e-13
    assert np.linalg.cond(Y[:4, :4]) < 100


def test_sign_fix_only_reads_leading_block():
    Q = rand_orth(30, 5, 9)
    s1 = R.sign_fix(Q)
    _, _, s2 = R.modified_lu(Q)
    assert np.array_equal(s1, s2)
