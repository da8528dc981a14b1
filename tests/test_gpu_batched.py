"""Batched refinement (eigref_refine_batched): many dense problems of uneven n
and k in one graph-replayed launch sequence.  Each problem must come out
exactly as it does from its own eigref_refine_dense call (same kernels, same
order of operations), match the FP64 oracle sweep by sweep, and stop on its
own schedule."""
import numpy as np
import pytest

from oracle import refine as R
from tests.gpu_util import dev, host, rel_diff, sweep_tol, U
from workloads import configs as C

pytestmark = pytest.mark.gpu

# uneven sizes, ragged against every tile (k = 64 is the batched workload's largest)
SHAPES = [(96, 4), (130, 7), (257, 16), (300, 33), (512, 64), (200, 12), (384, 5)]


@pytest.fixture(scope="module")
def eig():
    import paper_2602_23778_gb300 as pkg
    h = pkg.Handle(0)
    yield h
    h.close()


@pytest.fixture(scope="module")
def problems():
    return [C.config5_problem(i, n, k, seed=5100) for i, (n, k) in enumerate(SHAPES)]


def batch_inputs(ps):
    return [{"A": dev(p.A), "X": dev(np.asfortranarray(p.X0)), "target": "shift", "shift": p.shift,
             "norm_a": p.normA} for p in ps]


def test_fp64_batch_equals_single_calls(eig, problems):
    items = batch_inputs(problems)
    st, reps = eig.refine_batched(items, max_iters=6, precision="fp64")
    assert st == 0
    for p, it, rep in zip(problems, items, reps):
        X = dev(np.asfortranarray(p.X0))
        r1 = eig.refine_dense(dev(p.A), X, max_iters=6, norm_a=p.normA, target="shift", shift=p.shift)
        assert rep["status"] == 0 and rep["iterations"] == r1["iterations"] == 6
        assert np.array_equal(host(it["X"]), host(X)), (p.n, p.k)
        assert np.array_equal(rep["eigenvalues"], r1["eigenvalues"])


def test_fp64_batch_matches_oracle(eig, problems):
    items = batch_inputs(problems)
    st, reps = eig.refine_batched(items, max_iters=3, precision="fp64")
    assert st == 0
    for p, it, rep in zip(problems, items, reps):
        Xo, ro = R.refine(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, max_iters=3)
        tol = sweep_tol(p.normA + abs(p.shift), p.min_gap)
        assert rel_diff(host(it["X"]), Xo) <= tol, (p.n, p.k)
        assert rel_diff(rep["eigenvalues"], ro["d"]) <= 1e-12


def test_split_batch_matches_oracle(eig, problems):
    """The split form with the GPU shared between problems (no product split-K,
    shorter Gram split-K) still tracks the FP64 oracle within the split-form
    sweep bound."""
    items = batch_inputs(problems)
    st, reps = eig.refine_batched(items, max_iters=2, precision="bf16")
    assert st == 0
    for p, it, rep in zip(problems, items, reps):
        Xo, ro = R.refine(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, max_iters=2)
        tol = sweep_tol((1 + p.n ** 0.5 * 2.0 ** -56 / U) * (p.normA + abs(p.shift)), p.min_gap)
        assert rep["iterations"] == 2
        assert rel_diff(host(it["X"]), Xo) <= tol, (p.n, p.k)


def test_split_batch_equals_single_split_calls(eig, problems):
    """The grouped launches split K differently from a single call (no product
    split-K, shorter Gram split-K), but the split partials are exact int64 sums
    and every reduction order is fixed per problem: the results are the same
    bits."""
    items = batch_inputs(problems)
    st, reps = eig.refine_batched(items, max_iters=4, precision="bf16")
    assert st == 0
    for p, it, rep in zip(problems, items, reps):
        X = dev(np.asfortranarray(p.X0))
        r1 = eig.refine_dense(dev(p.A), X, max_iters=4, norm_a=p.normA, target="shift", shift=p.shift,
                              precision="bf16")
        assert np.array_equal(host(it["X"]), host(X)), (p.n, p.k, rep["ksplit"], r1["ksplit"])


def test_problems_stop_on_their_own_schedules(eig):
    """Problems that meet tol at different sweeps stop there; the others run on.
    Each stops where its own single call stops, with the same X."""
    ps = []
    for i, (n, k, noise) in enumerate([(200, 6, 1e-4), (333, 9, 1e-9), (150, 3, 1e-6)]):
        lam = C.separated_graded(n, k, 6100 + i, gap=0.05, tail=0.3)
        ps.append(C.householder(n, 8, k, lam, 6100 + i, target="largest_mag", x_noise=noise))
    items = batch_inputs(ps)
    kw = dict(max_iters=60, tol=1e-14, stop="residual", precision="fp64", check_every=4)
    st, reps = eig.refine_batched(items, **kw)
    assert st == 0
    its = [r["iterations"] for r in reps]
    assert len(set(its)) > 1, its
    for p, it, rep in zip(ps, items, reps):
        X = dev(np.asfortranarray(p.X0))
        r1 = eig.refine_dense(dev(p.A), X, norm_a=p.normA, target="shift", shift=p.shift, **kw)
        assert rep["iterations"] == r1["iterations"]
        assert rep["final_rel_residual"] <= 1e-14
        assert np.array_equal(host(it["X"]), host(X))


def test_batch_reports_the_failing_problem(eig, problems):
    """A problem that diverges is reported as such; the rest finish normally."""
    ps = problems[:3]
    items = batch_inputs(ps)
    # a random start for problem 1: ||E|| is O(1) at once, the divergence rule fires
    rnd = np.asfortranarray(np.linalg.qr(np.random.default_rng(7).standard_normal((ps[1].n, ps[1].k)))[0])
    items[1]["X"] = dev(rnd)
    st, reps = eig.refine_batched(items, max_iters=5, precision="fp64", raise_on_error=False)
    assert reps[0]["status"] == 0 and reps[2]["status"] == 0
    assert reps[1]["status"] != 0
    assert st == reps[1]["status"]
    assert "problem 1" in eig.last_error()


def test_batch_rejects_host_memory_and_leaves_x(eig, problems):
    import paper_2602_23778_gb300 as pkg
    p = problems[0]
    items = batch_inputs(problems[:2])
    x_before = host(items[0]["X"]).copy()
    items[1]["X"] = np.asfortranarray(p.X0.copy())  # host array: rejected
    items[1]["A"] = p.A
    with pytest.raises(pkg.EigrefError):
        eig.refine_batched(items, max_iters=2)
    assert np.array_equal(host(items[0]["X"]), x_before)


def test_split_batch_spanning_several_launch_groups(eig):
    """More problems than one grouped tensor-core launch holds (40), with
    k = 1 and odd sizes among them: every problem still matches the oracle."""
    shapes = [(96 + 37 * (i % 7), 1 + (5 * i) % 23) for i in range(45)]
    ps = [C.config5_problem(i, n, k, seed=5200) for i, (n, k) in enumerate(shapes)]
    items = batch_inputs(ps)
    st, reps = eig.refine_batched(items, max_iters=2, precision="bf16")
    assert st == 0
    for p, it, rep in zip(ps, items, reps):
        Xo, ro = R.refine(R.dense_operator(p.A, p.shift), p.X0, p.normA, p.shift, max_iters=2)
        tol = sweep_tol((1 + p.n ** 0.5 * 2.0 ** -56 / U) * (p.normA + abs(p.shift)), p.min_gap)
        assert rep["iterations"] == 2
        assert rel_diff(host(it["X"]), Xo) <= tol, (p.n, p.k)
