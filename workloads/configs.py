"""The five synthetic workloads (dense Householder-Q matrices, the 2-D
Laplacian, and a batch of uneven dense problems), seeded, with the data layout
both the oracle and the GPU path consume:

* ``A``: n x n FP64, C order (symmetric, so it is also its own column-major form)
* ``X0``: n x k FP64, Fortran order (column j = approximate eigenvector j)
* ``Xtrue``: the exact eigenvectors of the construction, same layout
* ``normA``: the spectral norm (max |lambda|), exact from the construction
* ``shift``: alpha of the shifted operator B = A - alpha I (0: no shift)

Holds no arithmetic of the refinement: the shift formulas below are the
paper's choice of alpha (Section 5.1), evaluated on the known spectrum.
"""
import numpy as np

from . import rng
from .dense import HouseholderProblem, orthonormalise, fp32_round
from .laplacian import Laplacian2D


class Problem(dict):
    __getattr__ = dict.__getitem__


def _noise(seed, stream, shape, std):
    return std * rng.normal(seed, stream, int(np.prod(shape))).reshape(shape, order="F")


def evenly_spaced(n):
    return -1.0 + 2.0 * np.arange(n) / (n - 1)


def shift_largest(normA, lam_kp1):
    """alpha for the k algebraically largest: the mirror of Section 5.1's rule."""
    return (lam_kp1 - normA) / 2.0


def shift_smallest(normA, lam_kp1):
    """alpha = (||A|| + lambda_{k+1}) / 2 for the k smallest (Section 5.1)."""
    return (normA + lam_kp1) / 2.0


def shift_smallest_mag(normA, lam_kp1):
    """alpha = (||A||^2 + lambda_{k+1}^2) / 2 for the k smallest |lambda|
    through B = A^2 - alpha I (Section 5.2; the midpoint of the squared
    spectrum's range above the targets)."""
    return (normA * normA + lam_kp1 * lam_kp1) / 2.0


def householder(n, m, k, lam, seed, target="largest_mag", x_noise=1e-7,
                noise_before_round=False, build_matrix=True):
    """Dense A = Q diag(lam) Q^T; target the k largest |lam| (no shift) or the
    k algebraically largest / smallest (shifted)."""
    hp = HouseholderProblem(n, m, lam, seed)
    if target == "largest_mag":
        order = np.argsort(-np.abs(lam), kind="stable")
    elif target == "largest":
        order = np.argsort(-lam, kind="stable")
    elif target == "smallest":
        order = np.argsort(lam, kind="stable")
    elif target == "smallest_mag":
        order = np.argsort(np.abs(lam), kind="stable")
    else:
        raise ValueError(target)
    idx = order[:k]
    lam_kp1 = lam[order[k]]
    normA = float(np.max(np.abs(lam)))
    shift = {"largest_mag": 0.0,
             "largest": shift_largest(normA, lam_kp1),
             "smallest": shift_smallest(normA, lam_kp1),
             "smallest_mag": shift_smallest_mag(normA, lam_kp1)}[target]
    Xt = hp.eigenvectors(idx)
    if noise_before_round:
        X0 = fp32_round(Xt + _noise(seed, 7, Xt.shape, x_noise))
    else:
        X0 = fp32_round(Xt) + _noise(seed, 7, Xt.shape, x_noise)
    X0 = orthonormalise(X0)
    lb = (lam * lam if target == "smallest_mag" else lam) - shift
    rest = np.delete(lb, idx)
    gamma = float(np.max(np.abs(rest)) / np.min(np.abs(lb[idx])))
    tl = lam[idx]
    gaps = np.abs(tl[:, None] - tl[None, :]) + np.eye(k) * 1e300
    return Problem(kind="dense", n=n, k=k, A=hp.matrix() if build_matrix else None,
                   X0=X0, Xtrue=Xt, lam=tl, lam_kp1=float(lam_kp1), normA=normA,
                   shift=float(shift), target=target, gamma=gamma,
                   min_gap=float(gaps.min()) if k > 1 else np.inf, gen=hp)


def config1(seed=1000):
    """n=512, k=8, 16 reflectors, lambda evenly spaced on [-1,1], the 8
    algebraically largest, X0 = orth(fp32(q + N(0,1e-6)))."""
    n = 512
    return householder(n, 16, 8, evenly_spaced(n), seed, target="largest",
                       x_noise=1e-6, noise_before_round=True)


def graded(n, seed):
    s = np.where(rng.uniform(seed, 3, n) < 0.5, -1.0, 1.0)
    return s * 10.0 ** (-6.0 * rng.uniform(seed, 4, n))


def config2(seed=2000, n=8192, k=64):
    """Graded spectrum sign * 10^(-6u), 64 reflectors, the 64 largest |lambda|."""
    return householder(n, 64, k, graded(n, seed), seed, target="largest_mag", x_noise=1e-7)


def separated_graded(n, k, seed, gap=1e-3, tail=0.8):
    """k target magnitudes 1 - gap*(i-1) and a graded tail tail*10^(-6u), random
    signs, placed at seeded random positions."""
    s = np.where(rng.uniform(seed, 3, n) < 0.5, -1.0, 1.0)
    mag = np.concatenate([1.0 - gap * np.arange(k),
                          tail * 10.0 ** (-6.0 * rng.uniform(seed, 4, n - k))])
    perm = np.argsort(rng.uint64(seed, 5, n), kind="stable")
    lam = np.empty(n)
    lam[perm] = s * mag
    return lam


def config3(seed=3000, n=16384, k=128, build_matrix=True):
    """n=16384, k=128, 64 reflectors, targets separated by >= 1e-3 ||A||."""
    return householder(n, 64, k, separated_graded(n, k, seed), seed,
                       target="largest_mag", x_noise=1e-7, build_matrix=build_matrix)


def config4(seed=4000, nx=1024, ny=1000, k=16, noise=1e-5, per_column=False):
    """Anisotropic Laplacian, the 16 smallest via the shift of Section 5.1.
    noise: std of the per-entry N(0, noise^2) perturbation; per_column=True
    scales it by 1/sqrt(n) (a column error of about ``noise``)."""
    L = Laplacian2D(nx, ny)
    n = L.n
    pqs = L.smallest(k + 1)
    Xt = np.asfortranarray(np.stack([L.eigenvector(pq) for pq in pqs[:k]], axis=1))
    std = noise / np.sqrt(n) if per_column else noise
    X0 = orthonormalise(fp32_round(Xt) + _noise(seed, 7, Xt.shape, std))
    lam = np.array([L.eigenvalue(pq) for pq in pqs])
    normA = float(L.norm_inf())
    shift = shift_smallest(normA, lam[k])
    row_ptr, col, val = L.csr()
    return Problem(kind="csr", n=n, k=k, row_ptr=row_ptr, col_idx=col, val=val,
                   X0=X0, Xtrue=Xt, lam=lam[:k], lam_kp1=float(lam[k]), normA=normA,
                   shift=float(shift), target="smallest", gen=L)


def config5_shapes(seed=5000, count=256):
    """(n, k) of the batched workload: n log-uniform on [256, 4096], k uniform
    on {4..64}."""
    u = rng.uniform(seed, 11, count)
    ns = np.rint(np.exp(np.log(256) + u * (np.log(4096) - np.log(256)))).astype(int)
    ks = 4 + (rng.uint64(seed, 12, count) % np.uint64(61)).astype(int)
    return list(zip(ns.tolist(), ks.tolist()))


def config5_problem(i, n, k, seed=5000):
    return householder(n, 16, k, evenly_spaced(n), seed * 1000 + i, target="largest",
                       x_noise=0.0)
