"""The split form of the Gram products for k <= 16 (CSR matrices): stacked BF16
digit planes on the tensor cores.  Entries against double-double dot
products within the slicing bound, exactness on all-positive inputs, many
splits (128-bit reduction), and refinement sweeps against the oracle."""
import numpy as np
import pytest

from oracle import dd, refine as R
from tests.gpu_util import dev, host, rel_diff, sweep_tol, U
from workloads import configs as C

pytestmark = pytest.mark.gpu

SLICES = 8


@pytest.fixture(scope="module")
def eig():
    import paper_2602_23778_gb300 as pkg
    h = pkg.Handle(0)
    yield h
    h.close()


def gram(eig, X, P, precision="bf16"):
    k = X.shape[1]
    G = np.zeros((k, k), order="F")
    S = np.zeros((k, k), order="F")
    eig.gram(dev(np.asfortranarray(X)), dev(np.asfortranarray(P)), G, S, precision=precision)
    return G, S


def bound(X, Y):
    """|error| of entry (i, j) of X^T Y: the rounded magnitudes and the
    truncated digit pairs (n (S + 2) 2^(e_i + f_j) 2^-8S over the sum,
    exponents of the column maxima) plus one FP64 rounding."""
    n = X.shape[0]
    e = np.frexp(np.abs(X).max(axis=0))[1]
    f = np.frexp(np.abs(Y).max(axis=0))[1]
    trunc = n * (SLICES + 2) * np.ldexp(1.0, e[:, None] + f[None, :] - 8 * SLICES)
    return trunc + 2 * U * (np.abs(X).T @ np.abs(Y))


def exact(X, Y):
    k1, k2 = X.shape[1], Y.shape[1]
    out = np.empty((k1, k2))
    for i in range(k1):
        for j in range(k2):
            hi, lo = dd.dot(X[:, i], Y[:, j])
            out[i, j] = hi + lo
    return out


@pytest.mark.parametrize("n,k", [(300, 1), (1000, 5), (5000, 16), (777, 13)])
def test_split_gram_vs_double_double(eig, n, k):
    rng = np.random.default_rng(n + k)
    X = rng.standard_normal((n, k)) * np.logspace(0, -3, k)[None, :]
    P = rng.standard_normal((n, k)) * 7.0
    G, S = gram(eig, X, P)
    assert np.all(np.abs(G - exact(X, X)) <= bound(X, X))
    assert np.all(np.abs(S - exact(X, P)) <= bound(X, P))
    G64, S64 = gram(eig, X, P, "fp64")
    assert rel_diff(G, G64) <= 1e-13 and rel_diff(S, S64) <= 1e-13


def test_split_gram_all_positive_is_exact(eig):
    """Every digit product of a weight group has the same sign: the partial
    sums grow linearly, the worst case for the FP32 chunks (960 deep)."""
    rng = np.random.default_rng(3)
    n, k = 200_000, 16
    X = rng.random((n, k))
    P = rng.random((n, k))
    G, S = gram(eig, X, P)
    assert np.all(np.abs(G - exact(X, X)) <= bound(X, X))
    assert np.all(np.abs(S - exact(X, P)) <= bound(X, P))
    assert (np.abs(S - exact(X, P)) / np.abs(exact(X, P))).max() < 8 * U


def test_split_gram_many_rows_many_splits(eig):
    """n = 1,100,000: many CTAs and chunks, the 128-bit sum over splits."""
    rng = np.random.default_rng(4)
    n, k = 1_100_000, 16
    X = rng.standard_normal((n, k)) / np.sqrt(n)
    P = rng.standard_normal((n, k))
    G, S = gram(eig, X, P)
    rows = [0, 3, 7, 15]
    Xs = X[:, rows]
    assert np.all(np.abs(G[np.ix_(rows, rows)] - exact(Xs, Xs)) <= bound(X, X)[np.ix_(rows, rows)])
    assert np.all(np.abs(S[np.ix_(rows, rows)] - exact(Xs, P[:, rows])) <= bound(X, P)[np.ix_(rows, rows)])


def laplace_case(nx, ny, k, seed=4000):
    return C.config4(seed=seed, nx=nx, ny=ny, k=k, noise=1e-5, per_column=True)


def split_tol(p):
    gaps = np.diff(np.sort(p.lam))
    return sweep_tol((1 + p.n ** 0.5 * 2.0 ** -(8 * SLICES - 8) / U) * (p.normA + abs(p.shift)),
                     gaps.min() if gaps.size else np.inf)


@pytest.mark.parametrize("nx,ny,k", [(40, 30, 16), (33, 17, 5), (64, 64, 1), (50, 41, 12), (37, 29, 2)])
def test_csr_split_sweeps_match_oracle(eig, nx, ny, k):
    p = laplace_case(nx, ny, k)
    X = dev(np.asfortranarray(p.X0))
    rg = eig.refine_csr(dev(p.row_ptr), dev(p.col_idx), dev(p.val), X, norm_a=p.normA, target="shift",
                        shift=p.shift, max_iters=3, precision="bf16")
    Xo, ro = R.refine(R.csr_operator(p.row_ptr, p.col_idx, p.val, p.n, p.shift), p.X0, p.normA, p.shift,
                      max_iters=3)
    assert rg["iterations"] == 3
    assert rel_diff(host(X), Xo) <= 3 * split_tol(p)
    # Rayleigh quotients of B = A - shift I, relative to ||B|| (the eigenvalues
    # of A are these plus the shift: small ones lose digits to the cancellation)
    assert np.abs(rg["eigenvalues"] - ro["d"]).max() <= 1e-12 * (p.normA + abs(p.shift))


def test_csr_split_full_size_sweep(eig):
    p = C.config4(per_column=True)
    X = dev(np.asfortranarray(p.X0))
    rg = eig.refine_csr(dev(p.row_ptr), dev(p.col_idx), dev(p.val), X, norm_a=p.normA, target="shift",
                        shift=p.shift, max_iters=1, precision="bf16")
    Xo, ro = R.refine(R.csr_operator(p.row_ptr, p.col_idx, p.val, p.n, p.shift), p.X0, p.normA, p.shift,
                      max_iters=1)
    assert rel_diff(host(X), Xo) <= split_tol(p)


def test_csr_split_needs_k_at_most_16(eig):
    import paper_2602_23778_gb300 as pkg
    p = laplace_case(30, 20, 17)
    with pytest.raises(pkg.EigrefError):
        eig.refine_csr(dev(p.row_ptr), dev(p.col_idx), dev(p.val), dev(np.asfortranarray(p.X0)),
                       norm_a=p.normA, target="shift", shift=p.shift, max_iters=1, precision="bf16")
