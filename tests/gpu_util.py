"""Helpers for the GPU tests: device copies in the layouts the C ABI takes,
and the parity measures.  Imports torch lazily so CPU-only collection works."""
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
    max(1e-12, 64 u ||B|| / min_gap)."""
    return max(1e-12, 64 * U * norm_b / min_gap)
