"""The bounded device waits run out without faulting anything: with a wait
limit of 1 ns every tensor-core kernel gives up at its first wait that is not
already complete, records EIGREF_E_TIMEOUT in the device status, releases its
tensor memory and returns; the call reports the status with X at the last
completed iterate, and the same handle then completes a normal call.  (The
failure is made on the host, by the limit; nothing here traps or hangs.)"""
import numpy as np
import pytest

from oracle import refine as R
from tests.gpu_util import dev, host, rel_diff, sweep_tol
from workloads import configs as C

pytestmark = pytest.mark.gpu

E_TIMEOUT = 8


@pytest.fixture(scope="module")
def eig():
    import paper_2602_23778_gb300 as pkg
    h = pkg.Handle(0)
    yield h
    h.close()


@pytest.mark.parametrize("k", [8, 64])
def test_dense_split_form_times_out_and_recovers(eig, k):
    """k = 8: the 128 x 32 product; k = 64: the 128 x 64 product, whose
    accumulator groups are drained one by one."""
    lam = C.separated_graded(300, k, 41, gap=min(0.01, 0.4 / k), tail=0.5)
    p = C.householder(300, 8, k, lam, 41, target="largest_mag", x_noise=1e-6)
    X0 = np.asfortranarray(p.X0)
    kw = dict(norm_a=p.normA, target="shift", shift=p.shift, precision="bf16", autotune=False, history=True)
    X = dev(X0)
    r = eig.refine_dense(dev(p.A), X, max_iters=4, wait_limit_s=1e-9, raise_on_error=False, **kw)
    assert r["status"] == E_TIMEOUT, r
    it = r["iterations"]
    assert it < 4
    Xo, _ = R.refine(R.dense_operator(p.A, p.shift), X0, p.normA, p.shift, max_iters=it)
    Xt = host(X)
    if it == 0:
        assert np.array_equal(Xt, X0)
    else:
        assert rel_diff(Xt, Xo) <= sweep_tol(p.normA + abs(p.shift), p.min_gap)
    # the handle is still usable: the same call without the limit
    X2 = dev(X0)
    r2 = eig.refine_dense(dev(p.A), X2, max_iters=4, **kw)
    assert r2["status"] == 0 and r2["iterations"] == 4
    Xo4, _ = R.refine(R.dense_operator(p.A, p.shift), X0, p.normA, p.shift, max_iters=4)
    assert rel_diff(host(X2), Xo4) <= sweep_tol(p.normA + abs(p.shift), p.min_gap)


@pytest.mark.parametrize("k", [16, 5])
def test_csr_split_form_times_out_and_recovers(eig, k):
    p = C.config4(seed=4000, nx=40, ny=30, k=k, noise=1e-5, per_column=True)
    X0 = np.asfortranarray(p.X0)
    args = (dev(p.row_ptr), dev(p.col_idx), dev(p.val))
    kw = dict(norm_a=p.normA, target="shift", shift=p.shift, precision="bf16")
    X = dev(X0)
    r = eig.refine_csr(*args, X, max_iters=3, wait_limit_s=1e-9, raise_on_error=False, **kw)
    assert r["status"] == E_TIMEOUT, r
    if r["iterations"] == 0:
        assert np.array_equal(host(X), X0)
    X2 = dev(X0)
    r2 = eig.refine_csr(*args, X2, max_iters=3, **kw)
    assert r2["status"] == 0 and r2["iterations"] == 3
    op = R.csr_operator(p.row_ptr, p.col_idx, p.val, p.n, p.shift)
    Xo, _ = R.refine(op, X0, p.normA, p.shift, max_iters=3)
    gaps = np.diff(np.sort(p.lam)).min()
    assert rel_diff(host(X2), Xo) <= 3 * sweep_tol(p.normA + abs(p.shift), gaps)
