"""The pins bite: plant plausible mistakes in a copy of the oracle (on the CPU)
and check that the pin battery of one refinement step rejects every one of
them while accepting the oracle as written."""
import inspect
import types

import numpy as np
import pytest

from oracle import refine as R
from tests.oracle_cases import delta_tie, separated

MUTATIONS = {
    "diag_sign": ("E[i, j] = (1.0 - alpha[i]) / 2.0", "E[i, j] = (alpha[i] - 1.0) / 2.0"),
    "gap_order": ("V[i, j] / (d[j] - d[i])", "V[i, j] / (d[i] - d[j])"),
    "e21_sign": ("E[k:, :] = V[k:, :] / d[None, :]", "E[k:, :] = -V[k:, :] / d[None, :]"),
    "beta_sign": ("-(Xh[:, i] @ Xh[:, j]) / 2.0", "(Xh[:, i] @ Xh[:, j]) / 2.0"),
    "h_transposed": ("Xt = Xh + apply_h(Y, T, E)", "Xt = Xh + apply_ht(Y, T, E)"),
    "v_untransformed": ("V = apply_ht(Y, T, R)", "V = R"),
    "residual_sign": ("R = W - Xh * d[None, :]", "R = W + Xh * d[None, :]"),
    "rq_unscaled": ("d = np.einsum(\"ij,ij->j\", Xh, W) / alpha", "d = np.einsum(\"ij,ij->j\", Xh, W)"),
    "wy_t_untransposed": ("return B - Y @ (T.T @ (Y.T @ B))", "return B - Y @ (T @ (Y.T @ B))"),
    "alg1_sign": ("T = -np.linalg.solve(Y1.T, np.eye(k))", "T = np.linalg.solve(Y1.T, np.eye(k))"),
    "delta_u": ("U_FP64 = 2.0 ** -53 ", "U_FP64 = 2.0 ** -52 "),
    "delta_no_c": ("return c * norm_b * U_FP64", "return norm_b * U_FP64"),
    "delta_no_norm": ("return c * norm_b * U_FP64", "return c * U_FP64"),
    "tie_strict": ("elif abs(d[j] - d[i]) <= delta:", "elif abs(d[j] - d[i]) < delta:"),
}


def mutant(name):
    src = inspect.getsource(R)
    old, new = MUTATIONS[name]
    assert src.count(old) == 1, name
    mod = types.ModuleType("oracle_mutant_" + name)
    exec(compile(src.replace(old, new), mod.__name__, "exec"), mod.__dict__)
    return mod


def battery(mod):
    """The step pins of test_oracle_step, as one predicate."""
    c = separated()
    delta = mod.delta_threshold(c.normA)
    op = mod.dense_operator(c.A)
    eps = 1e-6
    try:
        # first-order decay of non-target components
        X = c.perturbed(eps, seed=3)
        Xn, _ = mod.refine_step(op, X, delta)
        before, after = c.V.T @ X, c.V.T @ Xn
        for j in range(c.k):
            pred = c.w[c.rest] / c.lam_t[j] * before[c.rest, j]
            if np.abs(after[c.rest, j] - pred).max() > 50 * eps ** 2:
                return False
        # quadratic contraction inside the target block, Rayleigh quotients
        X = c.perturbed(eps, seed=4, within=True)
        Xn, info = mod.refine_step(op, X, delta)
        Ct = (c.V.T @ Xn)[[int(np.argmin(np.abs(c.w - l))) for l in c.lam_t], :]
        if np.abs(Ct - np.diag(np.diag(Ct))).max() > 50 * eps ** 2:
            return False
        if np.abs(info.d - c.lam_t).max() > 50 * eps ** 2:
            return False
        # diagonal branch
        X = c.Vt * (1.0 + eps * np.array([1.0, -2.0, 3.0]))[None, :]
        Xn, _ = mod.refine_step(op, X, delta)
        if np.abs(np.linalg.norm(Xn, axis=0) - 1.0).max() > 50 * eps ** 2:
            return False
        # clustered branch
        S = np.array([[0.0, 1.0, -2.0], [1.0, 0.0, 0.5], [-2.0, 0.5, 0.0]])
        X = c.Vt @ (np.eye(3) + eps * S)
        Xn, _ = mod.refine_step(op, X, mod.delta_threshold(c.normA, 1e30))
        if np.abs(Xn.T @ Xn - np.eye(3)).max() > 50 * eps ** 2:
            return False
        # the threshold: a tie at exactly delta takes beta, one ulp more divides
        for units, beta_branch in ((10, True), (11, False)):
            B, X, norm_b = delta_tie(units)
            _, info = mod.refine_step(mod.dense_operator(B), X, mod.delta_threshold(norm_b))
            if (info.E[0, 1] == 0.0) != beta_branch:
                return False
    except (np.linalg.LinAlgError, FloatingPointError):
        return False
    return True


def test_battery_accepts_oracle():
    assert battery(R)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_battery_rejects_mutant(name):
    assert not battery(mutant(name))
