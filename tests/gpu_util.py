"""Helpers for the GPU tests: device copies in the layouts the C ABI takes,
the parity measures and bounds, and a recorder of the achieved parity.
Imports torch lazily so CPU-only collection works."""
import json
import os

import numpy as np

U = 2.0 ** -53


def torch():
    import torch as t
    return t


def dev(a):
    """numpy -> CUDA tensor; 2-D Fortran-order arrays stay column-major."""
    t = torch()
    a = np.asarray(a)
    if a.ndim == 2 and a.flags.f_contiguous and not a.flags.c_contiguous:
        return t.from_numpy(np.ascontiguousarray(a.T)).cuda().t()
    return t.from_numpy(np.ascontiguousarray(a)).cuda()


def host(x):
    return x.detach().cpu().numpy()


def rel_diff(a, b):
    a, b = np.asarray(a), np.asarray(b)
    return float(np.abs(a - b).max() / np.abs(b).max())


def sweep_tol(norm_b, min_gap):
    """Per-sweep parity bound between two FP64 evaluations of Algorithm 4 that
    differ only in summation order: the gap divisions of Eq. (Eoffdiag)
    amplify an O(u ||B||) difference in V by 1/gap, so the bound is
    max(1e-12, 64 u ||B|| / min_gap) -- 1e-12 wherever min_gap >= 7.1e-3 ||B||."""
    return max(1e-12, 64 * U * norm_b / min_gap)


def record(test, **values):
    """Append the achieved parity figures of a test (and their bounds) as one
    JSON line to the file named by EIGREF_PARITY_LOG; nothing when unset."""
    path = os.environ.get("EIGREF_PARITY_LOG")
    if not path:
        return
    row = {"test": test}
    for key, v in values.items():
        row[key] = v if isinstance(v, (str, int)) else float(v)
    with open(path, "a") as f:
        f.write(json.dumps(row) + "\n")


def oracle_spread(apply_b, X0, norm_a, shift=0.0, abs_b=None, draws=4, seed=7, **kw):
    """The oracle's own sensitivity to rounding at its inputs: the largest
    change of its per-sweep ||E_t||_F, ||R_t||_F / ||A|| and final X over
    `draws` runs in which X0 is perturbed by one unit roundoff (relative,
    entry by entry) and every product W = B X by u (|B| |X|)_ij, one unit of
    the forward error bound of an FP64 dot product (gamma_n sum_l |b_il x_lj|
    without its dimension factor n), i.e. the scale by which two valid FP64
    evaluations of B X may differ.  abs_b(X) returns |B| |X| (default
    |W| + |shift| |X|).  Two correct evaluations (the oracle and the GPU,
    whose products and Gram sums round differently) differ by about this
    much; where the quantity is well conditioned the spread is a few ulps of
    it, near convergence it is the whole rounding floor.  Returns a dict of
    arrays (hist_corr, hist_res per sweep; X the max over entries) and the
    unperturbed run ("base")."""
    from oracle import refine as R
    X0 = np.asarray(X0)
    Xb, base = R.refine(apply_b, X0, norm_a, shift, **kw)
    rng = np.random.default_rng(seed)
    sc, sr, sx = np.zeros_like(base["hist_corr"]), np.zeros_like(base["hist_res"]), 0.0
    for _ in range(draws):
        def op(X, rng=rng):
            W = apply_b(X)
            scale = abs_b(X) if abs_b is not None else np.abs(W) + abs(shift) * np.abs(X)
            return W + U * scale * rng.uniform(-1, 1, W.shape)
        Xp0 = np.asfortranarray(X0 * (1.0 + U * rng.uniform(-1, 1, X0.shape)))
        Xp, rp = R.refine(op, Xp0, norm_a, shift, **kw)
        m = min(len(rp["hist_corr"]), len(base["hist_corr"]))
        sc[:m] = np.maximum(sc[:m], np.abs(rp["hist_corr"][:m] - base["hist_corr"][:m]))
        sr[:m] = np.maximum(sr[:m], np.abs(rp["hist_res"][:m] - base["hist_res"][:m]))
        sx = max(sx, float(np.abs(Xp - Xb).max()))
    return {"hist_corr": sc, "hist_res": sr, "X": sx, "base": base}


def corr_bound(ref, spread, factor=8.0):
    """|GPU - oracle| bound for a per-sweep norm: 1e-12 relative, plus
    `factor` times the oracle's own rounding spread at that sweep."""
    return 1e-12 * np.abs(ref) + factor * spread


def abs_dense(A, shift=0.0):
    """|B| |X| for B = A - shift I (dense), for oracle_spread."""
    Aa = np.abs(np.asarray(A))
    return lambda X: Aa @ np.abs(X) + abs(shift) * np.abs(X)


def abs_csr(row_ptr, col_idx, val, n, shift=0.0):
    """|B| |X| for B = A - shift I (CSR), for oracle_spread."""
    import scipy.sparse as sp
    Aa = sp.csr_matrix((np.abs(val), col_idx, row_ptr), shape=(n, n))
    return lambda X: Aa @ np.abs(X) + abs(shift) * np.abs(X)
