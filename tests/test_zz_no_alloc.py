"""eigref_product_dense_noalloc: the FP64 product for callers that cannot
allocate device memory (inside a framework whose memory pool owns the device,
or on a path where an allocation's implicit synchronisation is not allowed).
Its scratch is a fixed array inside the library; the test checks, through the
C ABI, that two calls in a row give what eigref_product_dense gives, and that
requests beyond the fixed size are refused.  Collected last on purpose."""
import numpy as np
import pytest

from tests.gpu_util import dev, host, rel_diff
from workloads import configs as C

pytestmark = pytest.mark.gpu


def case(n, k, seed):
    lam = C.separated_graded(n, k, seed, gap=min(0.01, 0.4 / k), tail=0.5)
    return C.householder(n, 8, k, lam, seed, target="largest_mag", x_noise=1e-6)


def test_noalloc_matches_product_dense_twice():
    import torch
    import paper_2602_23778_gb300 as pkg
    s = torch.cuda.Stream()
    with pkg.Handle(0) as h:
        # the larger call first, so the second one runs over stale scratch
        for n, k, shift, seed in ((3000, 96, 0.375, 21), (700, 17, -0.5, 22)):
            p = case(n, k, seed)
            A = dev(p.A)
            X = dev(np.asfortranarray(p.X0))
            want = torch.zeros_like(X)
            h.product_dense(A, X, want, shift=shift)
            got = torch.full_like(X, np.nan)
            torch.cuda.synchronize()
            st = pkg.product_dense_noalloc(A, X, got, shift=shift, stream=s)
            s.synchronize()
            assert st == pkg.OK, pkg.status_string(st)
            assert rel_diff(host(got), host(want)) <= 1e-15


def test_noalloc_rejects_oversize_and_host_memory():
    import torch
    import paper_2602_23778_gb300 as pkg
    n, k = 8193, 128                     # n * k just above 2^20
    A = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    X = torch.zeros((k, n), dtype=torch.float64, device="cuda").t()
    P = torch.zeros_like(X)
    assert n * k > pkg.NOALLOC_MAX_ELEMS
    assert pkg.product_dense_noalloc(A, X, P) == pkg.E_INVALID
    small = case(200, 4, 23)
    Xh = np.asfortranarray(small.X0)
    Ph = np.zeros_like(Xh)
    assert pkg.product_dense_noalloc(dev(small.A), Xh, Ph) == pkg.E_INVALID
