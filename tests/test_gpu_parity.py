"""Parity of the CUDA path (through the C ABI) with the CPU oracle, element by
element on the same seeded inputs: single sweeps over several tiles with
ragged tails, the 10-sweep trajectory of the n = 512 workload, CSR sweeps,
the product against double-double, stopping / status semantics and the
full-size workloads on sampled or whole outputs."""
import numpy as np
import pytest

from oracle import dd, refine as R
from tests.gpu_util import abs_csr, abs_dense, corr_bound, dev, host, oracle_spread, record, rel_diff, sweep_tol, U
from tests.oracle_cases import delta_tie
from workloads import configs as C

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def eig():
    import torch
    assert torch.cuda.is_available()
    import paper_2602_23778_gb300 as pkg
    h = pkg.Handle(0)
    yield h
    h.close()


def dense_case(n, k, seed, m=8):
    # target magnitudes 1 - gap*i stay above 0.6 > the tail's 0.5: gamma <= 5/6
    lam = C.separated_graded(n, k, seed, gap=min(0.01, 0.4 / k), tail=0.5)
    return C.householder(n, m, k, lam, seed, target="largest_mag", x_noise=1e-6)


def run_gpu(h, p, **kw):
    A = dev(p.A)
    X = dev(np.asfortranarray(p.X0))
    rep = h.refine_dense(A, X, norm_a=p.normA, target="shift", shift=p.shift, history=True, **kw)
    return host(X), rep


def run_oracle(p, **kw):
    return R.refine(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, **kw)


def check_norms(name, rg, p, spread):
    """||R_t|| and ||E_t|| of every sweep against the oracle: 1e-12 relative
    plus 8x the oracle's own rounding spread at that sweep (oracle_spread).
    Records the achieved differences."""
    ro = spread["base"]
    m = len(ro["hist_corr"])
    dc = np.abs(rg["hist_corr"][:m] - ro["hist_corr"])
    dr = np.abs(rg["hist_residual"][:m] - ro["hist_res"])
    bc, br = corr_bound(ro["hist_corr"], spread["hist_corr"]), corr_bound(ro["hist_res"], spread["hist_res"])
    record(name, corr_abs=dc.max(), corr_rel=(dc / ro["hist_corr"]).max(), corr_bound_rel=(bc / ro["hist_corr"]).min(),
           res_rel=(dr / ro["hist_res"]).max(), res_bound_rel=(br / ro["hist_res"]).min(),
           corr_min=ro["hist_corr"].min())
    assert np.all(dc <= bc), (dc, bc)
    assert np.all(dr <= br), (dr, br)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
@pytest.mark.parametrize("n,k", [(96, 1), (130, 3), (300, 8), (517, 17), (700, 64), (1000, 128), (257, 128)])
def test_single_sweep_dense(eig, n, k, precision):
    p = dense_case(n, k, seed=100 + n + k)
    Xg, rg = run_gpu(eig, p, max_iters=1, precision=precision)
    sp = oracle_spread(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, abs_dense(p.A, p.shift), max_iters=1)
    Xo, ro = run_oracle(p, max_iters=1)
    assert rg["status"] == 0 and rg["iterations"] == 1
    tol = sweep_tol(p.normA + abs(p.shift), p.min_gap)
    dx = rel_diff(Xg, Xo)
    record("single_sweep_dense[%s-%d-%d]" % (precision, n, k), x_rel=dx, x_bound=tol,
           d_rel=rel_diff(rg["eigenvalues"], ro["d"]), min_gap=p.min_gap)
    assert dx <= tol
    assert rel_diff(rg["eigenvalues"], ro["d"]) <= 1e-12
    check_norms("single_sweep_dense_norms[%s-%d-%d]" % (precision, n, k), rg, p, sp)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_trajectory_n512(eig, precision):
    """The n = 512, k = 8 workload: all 10 sweeps agree with the oracle."""
    p = C.config1()
    Xg, rg = run_gpu(eig, p, max_iters=10, precision=precision)
    sp = oracle_spread(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, abs_dense(p.A, p.shift), max_iters=10)
    Xo, ro = run_oracle(p, max_iters=10)
    assert rg["iterations"] == 10
    record("trajectory_n512[%s]" % precision, x_rel=rel_diff(Xg, Xo), x_bound=1e-12,
           d_rel=rel_diff(rg["eigenvalues"], ro["d"]))
    assert rel_diff(Xg, Xo) <= 1e-12
    check_norms("trajectory_n512_norms[%s]" % precision, rg, p, sp)
    assert rel_diff(rg["eigenvalues"], ro["d"]) <= 1e-14


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_correction_norm_at_converged_iterate(eig, precision):
    """||E_t||_F at the rounding floor: the oracle's iterate after 80 sweeps
    (||E|| near 1e-15), then one sweep on both sides from that iterate.  The
    norm is formed from the explicit rows of E (no k x k expansion), so the
    two sides differ by the rounding floor the oracle shows itself."""
    p = dense_case(400, 6, seed=9)
    Xc, rc = run_oracle(p, max_iters=80)
    assert rc["hist_corr"][-1] < 1e-13
    q = C.Problem({**p, "X0": np.asfortranarray(Xc)})
    Xg, rg = run_gpu(eig, q, max_iters=1, precision=precision)
    sp = oracle_spread(R.dense_operator(q.A, q.shift), q.X0, q.normA, q.shift, abs_dense(q.A, q.shift), max_iters=1)
    Xo, _ = run_oracle(q, max_iters=1)
    assert rg["iterations"] == 1
    record("converged_iterate[%s]" % precision, x_rel=rel_diff(Xg, Xo), corr=rg["hist_corr"][0],
           corr_oracle=sp["base"]["hist_corr"][0], corr_spread=sp["hist_corr"][0])
    check_norms("converged_iterate_norms[%s]" % precision, rg, q, sp)
    assert rel_diff(Xg, Xo) <= sweep_tol(q.normA + abs(q.shift), q.min_gap)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
def test_delta_tie_on_gpu(eig, precision):
    """The cluster threshold of Algorithm 4 on the GPU: Rayleigh quotients exactly delta
    apart take the beta branch (the sweep stays finite and small, as the
    oracle's), one ulp more takes the division (|E| huge: both report
    divergence after the first sweep)."""
    for units, want in ((10, 0), (11, 5)):
        B, X0, norm_b = delta_tie(units)
        X = dev(np.asfortranarray(X0))
        rg = eig.refine_dense(dev(B), X, norm_a=norm_b, max_iters=1, history=True, precision=precision,
                              raise_on_error=False)
        Xo, ro = R.refine(R.dense_operator(B), X0, norm_b, max_iters=1)
        assert ro["status"] == want and rg["status"] == want, (units, rg["status"], ro["status"])
        assert rg["iterations"] == ro["iterations"] == 1
        c_g, c_o = rg["hist_corr"][0], ro["hist_corr"][0]
        record("delta_tie[%s-%d]" % (precision, units), corr_rel=abs(c_g - c_o) / c_o, x_rel=rel_diff(host(X), Xo))
        assert abs(c_g - c_o) <= 1e-12 * c_o
        assert rel_diff(host(X), Xo) <= 1e-12
        assert (c_o < 1.0) == (want == 0)


def test_graph_and_chunking_do_not_change_results(eig):
    p = dense_case(300, 8, seed=7)
    X1, r1 = run_gpu(eig, p, max_iters=9, check_every=4)
    X2, r2 = run_gpu(eig, p, max_iters=9, use_graph=False, check_every=2)
    X3, r3 = run_gpu(eig, p, max_iters=9, check_every=64)
    assert r1["iterations"] == r2["iterations"] == r3["iterations"] == 9
    assert np.array_equal(X1, X2) and np.array_equal(X1, X3)


def test_stop_on_tolerance_matches_oracle(eig):
    p = dense_case(300, 8, seed=8)
    _, full = run_oracle(p, max_iters=30)
    tol = full["hist_corr"][12] * 1.0000001
    Xg, rg = run_gpu(eig, p, max_iters=30, tol=tol, check_every=8)
    Xo, ro = run_oracle(p, max_iters=30, tol=tol)
    assert ro["status"] == 0 and rg["status"] == 0
    assert rg["iterations"] == ro["iterations"] == 13
    assert rel_diff(Xg, Xo) <= 1e-12


def test_residual_criterion_and_accuracy(eig):
    """Converged: angle to the construction's eigenvectors and orthogonality
    in double-double, residual O(u) ||A|| (Section 4.2)."""
    p = dense_case(400, 6, seed=9)
    # the relative residual settles near 1e-15 here (rounding of B X); stop just above it
    Xg, rg = run_gpu(eig, p, max_iters=400, tol=3e-15, stop="residual")
    assert rg["status"] == 0, rg
    assert dd.sin_angles(Xg, p.Xtrue).max() < 1e-13
    assert np.abs(dd.orth_error(Xg)).max() < 1e-14
    _, res = dd.residual_dense(p.A, Xg)
    assert res.max() < 20 * U * p.normA


def test_not_converged_and_zero_iters(eig):
    p = dense_case(200, 4, seed=10)
    Xg, rg = run_gpu(eig, p, max_iters=3, tol=1e-16)
    assert rg["status"] == 6 and rg["iterations"] == 3
    X0 = dev(np.asfortranarray(p.X0))
    r = eig.refine_dense(dev(p.A), X0, max_iters=0)
    assert r["status"] == 0 and r["iterations"] == 0
    assert np.array_equal(host(X0), p.X0)


def test_nonfinite_keeps_last_finite(eig):
    p = dense_case(200, 4, seed=11)
    X0 = np.asfortranarray(p.X0.copy())
    X0[50, 2] = np.nan
    X = dev(X0)
    r = eig.refine_dense(dev(p.A), X, norm_a=p.normA, max_iters=5, raise_on_error=False)
    assert r["status"] == 7 and r["iterations"] == 0
    Xh = host(X)
    assert np.array_equal(np.isnan(Xh), np.isnan(X0))
    assert np.array_equal(Xh[~np.isnan(Xh)], X0[~np.isnan(X0)])


def test_invalid_arguments_leave_x_untouched(eig):
    import paper_2602_23778_gb300 as pkg
    p = dense_case(64, 4, seed=12)
    X = dev(np.asfortranarray(p.X0))
    A = dev(p.A)
    for kw in (dict(max_iters=-1), dict(tol=-1.0), dict(stop=7), dict(target=9)):
        with pytest.raises(pkg.EigrefError) as e:
            eig.refine_dense(A, X, **kw)
        assert e.value.status == 1
    assert np.array_equal(host(X), p.X0)
    big = dev(np.asfortranarray(np.zeros((64, 129))))
    with pytest.raises(pkg.EigrefError):
        eig.refine_dense(dev(np.eye(64)), big)


def test_host_buffers_match_device(eig):
    """Host A and X give the device-buffer results bit for bit; the handle's
    staging buffer for host A is reused by a smaller A, grown for a larger
    one and reused again (both forms)."""
    for n, k, seed in ((300, 5, 13), (200, 3, 16), (520, 33, 17), (300, 5, 13)):
        p = dense_case(n, k, seed=seed)
        for prec in ("fp64", "bf16"):
            Xd = dev(np.asfortranarray(p.X0))
            eig.refine_dense(dev(p.A), Xd, norm_a=p.normA, target="shift", shift=p.shift, max_iters=4,
                             precision=prec)
            Xh = np.asfortranarray(p.X0.copy())
            rh = eig.refine_dense(np.ascontiguousarray(p.A), Xh, norm_a=p.normA, target="shift", shift=p.shift,
                                  max_iters=4, precision=prec)
            assert rh["iterations"] == 4
            assert np.array_equal(Xh, host(Xd)), (n, k, prec)


def test_norm_inf_and_shift_targets(eig):
    """||A||_inf on the device and the shift of Section 5.1 (smallest)."""
    lam = np.linspace(-1, 1, 256)
    p = C.householder(256, 8, 4, lam, seed=14, target="smallest", x_noise=1e-7)
    X = dev(np.asfortranarray(p.X0))
    r = eig.refine_dense(dev(p.A), X, target="smallest", shift=p.lam_kp1, max_iters=2)
    ninf = np.abs(p.A).sum(1).max()
    assert abs(r["norm_a"] - ninf) <= 1e-14 * ninf
    assert abs(r["shift"] - 0.5 * (ninf + p.lam_kp1)) <= 1e-15 * ninf
    op = R.dense_operator(p.A, r["shift"])
    Xo, ro = R.refine(op, p.X0, ninf, r["shift"], max_iters=2)
    assert rel_diff(host(X), Xo) <= 1e-12


def test_product_dense_vs_double_double(eig):
    import torch
    p = dense_case(1000, 40, seed=15)
    A = dev(p.A)
    X = dev(np.asfortranarray(p.X0))
    P = torch.zeros_like(X)
    eig.product_dense(A, X, P, shift=0.25)
    Ph = host(P)
    rng = np.random.default_rng(0)
    rows, cols = rng.integers(0, 1000, 400), rng.integers(0, 40, 400)
    hi, lo = dd.product_entries(p.A, p.X0, rows, cols, shift=0.25)
    bound = 1000 * U * (np.abs(p.A) @ np.abs(p.X0) + 0.25 * np.abs(p.X0))
    assert np.all(np.abs(Ph[rows, cols] - hi) <= bound[rows, cols])


def laplace_case(nx, ny, k, noise, per_column, seed=4000):
    return C.config4(seed=seed, nx=nx, ny=ny, k=k, noise=noise, per_column=per_column)


def run_gpu_csr(h, p, **kw):
    X = dev(np.asfortranarray(p.X0))
    rep = h.refine_csr(dev(p.row_ptr), dev(p.col_idx), dev(p.val), X, norm_a=p.normA, target="shift",
                       shift=p.shift, history=True, **kw)
    return host(X), rep


def run_oracle_csr(p, **kw):
    op = R.csr_operator(p.row_ptr, p.col_idx, p.val, p.n, p.shift)
    return R.refine(op, p.X0, p.normA, p.shift, **kw)


@pytest.mark.parametrize("precision", ["fp64", "bf16"])
@pytest.mark.parametrize("nx,ny,k", [(40, 30, 16), (33, 17, 5), (64, 64, 3)])
def test_csr_sweeps(eig, nx, ny, k, precision):
    p = laplace_case(nx, ny, k, noise=1e-5, per_column=True)
    Xg, rg = run_gpu_csr(eig, p, max_iters=3, precision=precision)
    Xo, ro = run_oracle_csr(p, max_iters=3)
    assert rg["iterations"] == 3
    gaps = np.diff(np.sort(p.lam)).min()
    tol = sweep_tol(p.normA + abs(p.shift), gaps) * 3
    record("csr_sweeps[%s-%d-%d-%d]" % (precision, nx, ny, k), x_rel=rel_diff(Xg, Xo), x_bound=tol)
    assert rel_diff(Xg, Xo) <= tol
    op = R.csr_operator(p.row_ptr, p.col_idx, p.val, p.n, p.shift)
    check_norms("csr_sweeps_norms[%s-%d-%d-%d]" % (precision, nx, ny, k), rg, p,
                oracle_spread(op, p.X0, p.normA, p.shift, abs_csr(p.row_ptr, p.col_idx, p.val, p.n, p.shift),
                              max_iters=3))


def test_csr_product_vs_scipy(eig):
    import torch
    import scipy.sparse as sp
    p = laplace_case(50, 41, 6, noise=1e-3, per_column=False)
    X = dev(np.asfortranarray(p.X0))
    P = torch.zeros_like(X)
    eig.product_csr(dev(p.row_ptr), dev(p.col_idx), dev(p.val), X, P, shift=p.shift)
    A = sp.csr_matrix((p.val, p.col_idx, p.row_ptr), shape=(p.n, p.n))
    ref = A @ p.X0 - p.shift * p.X0
    assert rel_diff(host(P), ref) <= 1e-15 * 16


def test_divergence_matches_oracle(eig):
    p = laplace_case(40, 38, 16, noise=3e-2, per_column=False)
    Xg, rg = run_gpu_csr(eig, p, max_iters=50, raise_on_error=False)
    Xo, ro = run_oracle_csr(p, max_iters=50)
    assert ro["status"] == 5 and rg["status"] == 5
    assert rg["iterations"] == ro["iterations"]


# ---- full-size workloads ---------------------------------------------------

@pytest.mark.slow
def test_full_size_n16384_k128_sweep(eig):
    p = C.config3()
    Xg, rg = run_gpu(eig, p, max_iters=1)
    Xo, ro = run_oracle(p, max_iters=1)
    assert rel_diff(Xg, Xo) <= sweep_tol(p.normA, p.min_gap)
    assert rel_diff(rg["eigenvalues"], ro["d"]) <= 1e-12


@pytest.mark.slow
def test_full_size_n8192_k64_sweeps(eig):
    p = C.config2()
    Xg, rg = run_gpu(eig, p, max_iters=2)
    Xo, ro = run_oracle(p, max_iters=2)
    assert rel_diff(Xg, Xo) <= sweep_tol(p.normA, p.min_gap)


@pytest.mark.slow
def test_full_size_laplacian_sweep(eig):
    p = C.config4()
    Xg, rg = run_gpu_csr(eig, p, max_iters=1)
    Xo, ro = run_oracle_csr(p, max_iters=1)
    gaps = np.diff(np.sort(p.lam)).min()
    assert rel_diff(Xg, Xo) <= sweep_tol(p.normA + abs(p.shift), gaps)
    assert abs(rg["hist_residual"][0] - ro["hist_res"][0]) <= 1e-9 * ro["hist_res"][0]
