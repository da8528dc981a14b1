"""ORACLE (test infrastructure only): closed forms of the convergence analysis
(Section 3.2 and Section 3.3), used to pin the oracle's measured behaviour."""
import numpy as np


def chi(eps):
    """chi(eps) = (3 - 2 eps) / (1 - eps)^2 (Section 3.2.1)."""
    return (3.0 - 2.0 * eps) / (1.0 - eps) ** 2


def eta(eps):
    """eta(eps) = 2 (1 + 2 eps + chi eps^2) chi / ((1 - eps)(1 - 2 eps - chi eps^2))."""
    c = chi(eps)
    return 2.0 * (1.0 + 2.0 * eps + c * eps ** 2) * c / ((1.0 - eps) * (1.0 - 2.0 * eps - c * eps ** 2))


def omega(eps):
    """omega(eps) = 2 chi + 2 eta eps + chi eta eps^2."""
    c, e = chi(eps), eta(eps)
    return 2.0 * c + 2.0 * e * eps + c * e * eps ** 2


def alpha_sufficient(rho1, rho2):
    """alpha of Theorem 3.6, Eq. (alpha): the largest ratio
    max_{j>k}|lambda| / min_{i<=k}|lambda| the sufficient condition admits."""
    r1, r2 = float(rho1) ** 2, float(rho2) ** 2
    return (r2 - 1.0) / r2 * (0.98 - 46.0 / (r1 - 1.0)) - 92.0 / r2


def gamma(lam_b, target_idx):
    """The linear rate gamma = max_{i>k} |lambda_{p_i}| / min_{j<=k} |lambda_{p_j}|
    (end of Section 3.2) for the eigenvalues lam_b of the refined operator."""
    lam_b = np.asarray(lam_b, dtype=np.float64)
    mask = np.zeros(lam_b.shape, bool)
    mask[np.asarray(target_idx)] = True
    return float(np.max(np.abs(lam_b[~mask])) / np.min(np.abs(lam_b[mask])))
