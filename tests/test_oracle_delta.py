"""Pins of the cluster threshold of Algorithm 4 (the choice between beta and
the gap division in E-tilde_L) against what Section
3.1.3 fixes: delta = c ||A|| u with c = 10 and u the unit roundoff of binary64
(2^-53), and the tie |d_j - d_i| = delta taking the beta branch (the test in
Algorithm 4 is "<= delta").  The Rayleigh quotients of the crafted cases are exact
binary64 numbers, so the two branches are decided exactly, one ulp apart."""
import numpy as np
import pytest

from oracle import refine as R
from tests.oracle_cases import delta_tie


def test_delta_value_is_c_norm_u():
    assert R.U_FP64 == 2.0 ** -53
    assert R.delta_threshold(1.0) == 10 * 2.0 ** -53
    assert R.delta_threshold(2.0) == 20 * 2.0 ** -53
    assert R.delta_threshold(3.0, 4.0) == 12 * 2.0 ** -53


def offdiag_e(gap_units):
    B, X, norm_b = delta_tie(gap_units)
    delta = R.delta_threshold(norm_b)
    _, info = R.refine_step(R.dense_operator(B), X, delta)
    assert info.d[1] - info.d[0] == gap_units * 2.0 ** -52   # exact quotients
    return info, delta


def test_tie_takes_beta_branch():
    """|d_1 - d_0| = delta exactly: E_01 = beta_01 = -x_0^T x_1 / 2 = 0."""
    info, delta = offdiag_e(10)
    assert info.d[1] - info.d[0] == delta
    assert info.E[0, 1] == 0.0 and info.E[1, 0] == 0.0


def test_one_ulp_above_takes_the_division():
    """|d_1 - d_0| = delta + 2^-52: E_01 = V_01 / (d_1 - d_0), V_01 = x_0^T r_1 = t."""
    info, delta = offdiag_e(11)
    gap = info.d[1] - info.d[0]
    assert gap > delta
    assert info.V[0, 1] == pytest.approx(2.0 ** -10, rel=1e-12)
    assert info.E[0, 1] == pytest.approx(info.V[0, 1] / gap, rel=1e-15)
    assert abs(info.E[0, 1]) > 1e10


def test_other_pairs_use_the_division():
    info, _ = offdiag_e(10)
    for i, j in ((0, 2), (2, 3), (1, 3)):
        assert info.E[i, j] == pytest.approx(info.V[i, j] / (info.d[j] - info.d[i]), rel=1e-15)
