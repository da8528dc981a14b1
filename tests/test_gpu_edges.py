"""Edge cases of the refinement calls: the smallest problems (n = 2, k = 1),
k = n - 1, the largest k (128), inputs that must be refused, and inputs that
make a sweep non-finite -- against the oracle where a result is defined."""
import numpy as np
import pytest

from oracle import refine as R
from tests.gpu_util import dev, host, rel_diff, sweep_tol, U
from workloads import configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eig():
    import paper_2602_23778_gb300 as pkg
    h = pkg.Handle(0)
    yield h
    h.close()


def small_problem(n, k, seed):
    """A = Q diag(lam) Q^T with a random orthogonal Q and magnitudes spread so
    that the k largest |lam| are separated from the rest."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(0.1, 1.0, n) * np.where(np.arange(n) % 2 == 0, 1.0, -1.0)
    A = (Q * lam[None, :]) @ Q.T
    A = 0.5 * (A + A.T)
    order = np.argsort(-np.abs(lam), kind="stable")
    Xt = Q[:, order[:k]]
    X0 = C.orthonormalise(Xt + 1e-6 * rng.standard_normal(Xt.shape))
    gaps = np.abs(np.diff(np.sort(lam[order[:k]]))) if k > 1 else np.array([np.inf])
    return A, X0, Xt, float(np.abs(lam).max()), float(gaps.min())


@pytest.mark.parametrize("n,k", [(2, 1), (3, 2), (17, 16), (33, 32), (129, 128)])
@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_smallest_and_widest_problems_match_oracle(eig, n, k, precision):
    A, X0, Xt, normA, gap = small_problem(n, k, seed=10 * n + k)
    X = dev(np.asfortranarray(X0))
    rg = eig.refine_dense(dev(A), X, max_iters=3, norm_a=normA, precision=precision)
    Xo, ro = R.refine(R.dense_operator(A), X0, normA, max_iters=3)
    assert rg["status"] == 0 and rg["iterations"] == 3
    tol = sweep_tol((1 + n ** 0.5 * 2.0 ** -56 / U) * normA, gap)
    assert rel_diff(host(X), Xo) <= 3 * tol


def test_k_above_the_limit_is_refused(eig):
    import paper_2602_23778_gb300 as pkg
    A, X0, _, normA, _ = small_problem(140, 129, seed=3)
    X = dev(np.asfortranarray(X0))
    with pytest.raises(pkg.EigrefError):
        eig.refine_dense(dev(A), X, max_iters=1, norm_a=normA)
    assert np.array_equal(host(X), X0)


def test_k_equal_n_is_refused(eig):
    import paper_2602_23778_gb300 as pkg
    A, X0, _, normA, _ = small_problem(8, 8, seed=4)
    with pytest.raises(pkg.EigrefError):
        eig.refine_dense(dev(A), dev(np.asfortranarray(X0)), max_iters=1, norm_a=normA)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_zero_column_is_reported_and_x_kept(eig, precision):
    """A zero column has no Rayleigh quotient (0 / 0): the sweep is non-finite,
    the call says so, and X keeps the last finite iterate (the input)."""
    import paper_2602_23778_gb300 as pkg
    A, X0, _, normA, _ = small_problem(200, 4, seed=5)
    X0 = X0.copy()
    X0[:, 2] = 0.0
    X = dev(np.asfortranarray(X0))
    rg = eig.refine_dense(dev(A), X, max_iters=3, norm_a=normA, precision=precision, raise_on_error=False)
    assert rg["status"] in (pkg.E_NONFINITE, pkg.E_SINGULAR_WY)
    assert rg["iterations"] == 0
    Xh = host(X)
    assert np.array_equal(Xh[:, [0, 1, 3]], X0[:, [0, 1, 3]])


def test_empty_csr_is_a_status_not_a_fault(eig):
    import torch
    import paper_2602_23778_gb300 as pkg
    n, k = 50, 2
    rp = torch.zeros(n + 1, dtype=torch.int32, device="cuda")
    ci = torch.zeros(0, dtype=torch.int32, device="cuda")
    val = torch.zeros(0, dtype=torch.float64, device="cuda")
    X = dev(np.asfortranarray(np.eye(n)[:, :k]))
    # no stored entries: refused as missing arrays, or (if the empty tensors
    # carry an address) a zero matrix, whose Rayleigh quotients 0 / 1 make the
    # gap divisions non-finite -- either way a status, never a fault
    rg = eig.refine_csr(rp, ci, val, X, max_iters=1, norm_a=1.0, raise_on_error=False)
    assert rg["status"] in (pkg.E_INVALID, pkg.E_NONFINITE)


def test_auto_precision_picks_the_form(eig):
    """precision = auto: the split form for dense 1024 <= n <= 2^18 (the report
    names its split-K), FP64 below; both within their sweep bounds."""
    for n, split in ((1500, True), (500, False)):
        A, X0, _, normA, gap = small_problem(n, 8, seed=n)
        X = dev(np.asfortranarray(X0))
        rg = eig.refine_dense(dev(A), X, max_iters=2, norm_a=normA, precision="auto")
        assert (rg["psplit"] > 0) == split
        Xo, _ = R.refine(R.dense_operator(A), X0, normA, max_iters=2)
        assert rel_diff(host(X), Xo) <= 2 * sweep_tol((1 + n ** 0.5 * 2.0 ** -56 / U) * normA, gap)


def as_csr(A):
    rows, cols = np.nonzero(A)
    row_ptr = np.zeros(A.shape[0] + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), cols.astype(np.int32), A[rows, cols].astype(np.float64)


@pytest.mark.parametrize("n,k", [(3, 2), (17, 16), (40, 4), (70, 10), (200, 14)])
def test_small_csr_split_form_matches_oracle(eig, n, k):
    """The CSR split form's kernels at sizes below one tile (n < 64 rows of a
    Gram block, n < 128 rows of an update tile) and with ragged last tiles,
    for even k (the Gram planes cut in shared memory, the tensor-core row
    update) -- against the oracle."""
    A, X0, Xt, normA, gap = small_problem(n, k, seed=20 * n + k)
    rp, ci, val = as_csr(A)
    X = dev(np.asfortranarray(X0))
    rg = eig.refine_csr(dev(rp), dev(ci), dev(val), X, max_iters=3, norm_a=normA, precision="bf16")
    Xo, ro = R.refine(R.dense_operator(A), X0, normA, max_iters=3)
    assert rg["status"] == 0 and rg["iterations"] == 3
    tol = sweep_tol((1 + n ** 0.5 * 2.0 ** -56 / U) * normA, gap)
    assert rel_diff(host(X), Xo) <= 3 * tol
