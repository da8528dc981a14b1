"""Python binding of the eigref C ABI (include/eigref.h): argument marshalling
only.  Every step of the refinement runs in the CUDA library
``_build/libeigref.so``; there is no Python or CPU fallback -- importing a
function that needs the library raises if it is not built.

Arrays may be torch tensors (CUDA or CPU) or numpy arrays.  Dense ``A`` is
n x n FP64 (any of C or Fortran order: it is symmetric); ``X`` is n x k FP64
column-major (numpy: Fortran order; torch: ``x.t().contiguous().t()``).
"""
import ctypes
import os

import numpy as np

from . import build as _build_mod

_LIB = None

OK, E_INVALID, E_CUDA, E_NOMEM, E_SINGULAR_WY, E_DIVERGED, E_NOT_CONVERGED, E_NONFINITE, E_TIMEOUT, \
    E_UNSUPPORTED = range(10)
TARGETS = {"largest_mag": 0, "largest": 1, "smallest": 2, "shift": 3, "smallest_mag": 4}
PRECISIONS = {"fp64": 0, "bf16": 1, "int8": 2, "auto": 3}
STOPS = {"correction": 0, "residual": 1}
BETAS = {"cluster": 0, "zero": 1}

SYMBOLS = ["eigref_params_default", "eigref_create", "eigref_destroy", "eigref_refine_dense",
           "eigref_refine_csr", "eigref_product_dense", "eigref_product_csr", "eigref_status_string",
           "eigref_last_error", "eigref_product_dense_noalloc", "eigref_refine_batched", "eigref_gram"]
NOALLOC_MAX_ELEMS = 1 << 20


class Params(ctypes.Structure):
    _fields_ = [("target", ctypes.c_int), ("shift", ctypes.c_double), ("norm_a", ctypes.c_double),
                ("max_iters", ctypes.c_int), ("tol", ctypes.c_double), ("stop", ctypes.c_int),
                ("precision", ctypes.c_int), ("slices", ctypes.c_int), ("beta", ctypes.c_int),
                ("delta_c", ctypes.c_double), ("div_factor", ctypes.c_double), ("div_floor", ctypes.c_double),
                ("check_every", ctypes.c_int), ("sign_fix", ctypes.c_int), ("use_graph", ctypes.c_int),
                ("profile", ctypes.c_int), ("rayleigh_ritz", ctypes.c_int), ("judge_cols", ctypes.c_int),
                ("reorth", ctypes.c_int), ("resign", ctypes.c_int), ("autotune", ctypes.c_int),
                ("wait_limit_s", ctypes.c_double), ("product_tile", ctypes.c_int)]


class Report(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("iterations", ctypes.c_int),
                ("final_rel_residual", ctypes.c_double), ("final_corr_norm", ctypes.c_double),
                ("shift", ctypes.c_double), ("norm_a", ctypes.c_double), ("delta", ctypes.c_double),
                ("setup_ms", ctypes.c_double), ("sweeps_ms", ctypes.c_double),
                ("eigenvalues", ctypes.POINTER(ctypes.c_double)),
                ("hist_residual", ctypes.POINTER(ctypes.c_double)),
                ("hist_corr", ctypes.POINTER(ctypes.c_double)),
                ("product_ms", ctypes.c_double), ("kernel_launches", ctypes.c_int64),
                ("product_launches", ctypes.c_int), ("psplit", ctypes.c_int), ("ksplit", ctypes.c_int)]


class Problem(ctypes.Structure):
    _fields_ = [("A", ctypes.c_void_p), ("n", ctypes.c_int64), ("lda", ctypes.c_int64),
                ("X", ctypes.c_void_p), ("ldx", ctypes.c_int64), ("k", ctypes.c_int),
                ("target", ctypes.c_int), ("shift", ctypes.c_double), ("norm_a", ctypes.c_double)]


class EigrefError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("eigref status %d: %s" % (status, msg))
        self.status = status


def library_path():
    return _build_mod.LIB


def lib():
    """The loaded CUDA library; raises if it has not been built."""
    global _LIB
    if _LIB is None:
        path = library_path()
        if not os.path.exists(path):
            raise ImportError("libeigref.so is not built (run paper_2602_23778_gb300.build.build() or "
                              "__graft_entry__.build()); there is no CPU fallback")
        L = ctypes.CDLL(path)
        vp, i64, i32, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.eigref_params_default.argtypes = [ctypes.POINTER(Params)]
        L.eigref_params_default.restype = None
        L.eigref_create.argtypes = [ctypes.POINTER(vp), i32, vp]
        L.eigref_destroy.argtypes = [vp]
        L.eigref_refine_dense.argtypes = [vp, vp, i64, i64, vp, i64, i32, ctypes.POINTER(Params),
                                          ctypes.POINTER(Report)]
        L.eigref_refine_csr.argtypes = [vp, vp, vp, vp, i64, i64, vp, i64, i32, ctypes.POINTER(Params),
                                        ctypes.POINTER(Report)]
        L.eigref_product_dense.argtypes = [vp, vp, i64, i64, vp, i64, i32, dbl, i32, i32, vp, i64]
        L.eigref_product_csr.argtypes = [vp, vp, vp, vp, i64, i64, vp, i64, i32, dbl, vp, i64]
        L.eigref_product_dense_noalloc.argtypes = [vp, i64, i64, vp, i64, i32, dbl, vp, i64, vp]
        L.eigref_refine_batched.argtypes = [vp, i32, ctypes.POINTER(Problem), ctypes.POINTER(Params),
                                            ctypes.POINTER(Report)]
        L.eigref_gram.argtypes = [vp, vp, i64, vp, i64, i64, i32, i32, i32, vp, vp]
        L.eigref_status_string.argtypes = [i32]
        L.eigref_status_string.restype = ctypes.c_char_p
        L.eigref_last_error.argtypes = [vp]
        L.eigref_last_error.restype = ctypes.c_char_p
        _LIB = L
    return _LIB


def status_string(s):
    return lib().eigref_status_string(int(s)).decode()


# ---- array marshalling ------------------------------------------------------

def sliced_info(precision, n, k, slices=8, product_tile=0):
    """Work of one split-precision product W = B X as the library pads it:
    S (S + 1) / 2 digit-plane pairs, each a 2 n_pad^2 k_pad-flop BF16 GEMM
    (n_pad = n rounded up to 256, k_pad = k rounded up to 32), and the kernel
    that runs it (128 x 64 tiles where k_pad is a multiple of 64, unless
    product_tile asks for 32)."""
    n_pad = -(-n // 256) * 256
    k_pad = -(-k // 32) * 32
    pairs = slices * (slices + 1) // 2
    wide = product_tile != 32 and k_pad % 64 == 0
    return {"kernel": "sliced_wide_kernel (128 x 64 tiles)" if wide else "sliced_mma_kernel (product mode)",
            "slices": slices, "pairs": pairs,
            "executed_flops": 2.0 * n_pad * n_pad * k_pad * pairs,
            "a_plane_bytes": 2.0 * slices * n_pad * n_pad}

def _same_shape(name, got, want):
    """Refuse an output or operand whose shape does not match before anything
    reaches the library (a narrow P would be written past its end)."""
    if tuple(got) != tuple(want):
        raise ValueError("%s is %s, expected %s" % (name, "x".join(map(str, got)), "x".join(map(str, want))))


def product_dense_noalloc(A, X, P, shift=0.0, stream=None):
    """P = (A - shift I) X through eigref_product_dense_noalloc: FP64, device
    arrays only, queued on ``stream`` (torch stream, raw handle or None) with
    no device allocation; returns the status code."""
    pa, n, lda, ka = _dense_a(A)
    px, nx, k, ldx, kx = _colmajor(X)
    pp, np_, kp, ldp, kpp = _colmajor(P, "P")
    _same_shape("X", (nx, k), (n, k))
    _same_shape("P", (np_, kp), (n, k))
    sp = None
    if stream is not None:
        sp = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    return lib().eigref_product_dense_noalloc(pa, n, lda, px, ldx, k, float(shift), pp, ldp, sp)



def _info(a):
    """(pointer, shape, strides in elements, dtype name, is_torch, keepalive)."""
    if type(a).__module__.startswith("torch"):
        return a.data_ptr(), tuple(a.shape), tuple(a.stride()), str(a.dtype).replace("torch.", ""), a
    a = np.asarray(a)
    return a.ctypes.data, a.shape, tuple(s // a.itemsize for s in a.strides), a.dtype.name, a


def _dense_a(A):
    p, shape, st, dt, keep = _info(A)
    if dt != "float64" or len(shape) != 2 or shape[0] != shape[1]:
        raise ValueError("A must be a square float64 matrix")
    if st[1] == 1:
        lda = st[0]
    elif st[0] == 1:
        lda = st[1]
    else:
        raise ValueError("A needs unit stride in one dimension")
    return p, shape[0], max(lda, 1), keep


def _colmajor(X, name="X"):
    p, shape, st, dt, keep = _info(X)
    if dt != "float64" or len(shape) != 2:
        raise ValueError("%s must be a 2-D float64 array" % name)
    n, k = shape
    if st[0] != 1 and n > 1:
        raise ValueError("%s must be column-major (numpy: np.asfortranarray; torch: x.t().contiguous().t())" % name)
    ld = st[1] if k > 1 else n
    return p, n, k, ld, keep


def _int32(a, name):
    p, shape, st, dt, keep = _info(a)
    if dt != "int32" or len(shape) != 1 or (len(shape) == 1 and shape[0] > 1 and st[0] != 1):
        raise ValueError("%s must be a contiguous int32 vector" % name)
    return p, shape[0], keep


def _f64vec(a, name):
    p, shape, st, dt, keep = _info(a)
    if dt != "float64" or len(shape) != 1 or (shape[0] > 1 and st[0] != 1):
        raise ValueError("%s must be a contiguous float64 vector" % name)
    return p, shape[0], keep


class Handle:
    """One eigref handle: a CUDA device, a stream and a workspace."""

    def __init__(self, device=0, stream=None):
        L = lib()
        h = ctypes.c_void_p()
        sp = None
        if stream is not None:
            sp = ctypes.c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
        st = L.eigref_create(ctypes.byref(h), int(device), sp)
        if st != OK:
            raise EigrefError(st, "eigref_create failed on device %d" % device)
        self._h = h

    def close(self):
        if getattr(self, "_h", None):
            lib().eigref_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def last_error(self):
        return lib().eigref_last_error(self._h).decode()

    @staticmethod
    def params(**kw):
        p = Params()
        lib().eigref_params_default(ctypes.byref(p))
        for key, v in kw.items():
            if key == "target":
                v = TARGETS[v] if isinstance(v, str) else v
            elif key == "precision":
                v = PRECISIONS[v] if isinstance(v, str) else v
            elif key == "stop":
                v = STOPS[v] if isinstance(v, str) else v
            elif key == "beta":
                v = BETAS[v] if isinstance(v, str) else v
            elif key in ("sign_fix", "use_graph", "profile", "rayleigh_ritz", "reorth", "resign", "autotune"):
                v = int(bool(v))
            setattr(p, key, v)
        return p

    def _finish(self, st, rep, k, want, raise_on_error):
        out = dict(status=st, status_string=status_string(st), iterations=rep.iterations,
                   final_rel_residual=rep.final_rel_residual, final_corr_norm=rep.final_corr_norm,
                   shift=rep.shift, norm_a=rep.norm_a, delta=rep.delta, setup_ms=rep.setup_ms,
                   sweeps_ms=rep.sweeps_ms, product_ms=rep.product_ms, product_launches=rep.product_launches,
                   kernel_launches=rep.kernel_launches, psplit=rep.psplit, ksplit=rep.ksplit,
                   error=self.last_error())
        ev, hr, hc = want
        out["eigenvalues"] = ev
        if hr is not None:
            out["hist_residual"] = hr[:rep.iterations].copy()
            out["hist_corr"] = hc[:rep.iterations].copy()
        if raise_on_error and st in (E_INVALID, E_CUDA, E_NOMEM, E_UNSUPPORTED):
            raise EigrefError(st, out["error"])
        return out

    def _report(self, k, max_iters, history):
        rep = Report()
        ev = np.zeros(k)
        rep.eigenvalues = ev.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        hr = hc = None
        if history:
            hr, hc = np.zeros(max(1, max_iters)), np.zeros(max(1, max_iters))
            rep.hist_residual = hr.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            rep.hist_corr = hc.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        return rep, (ev, hr, hc)

    def refine_dense(self, A, X, history=False, raise_on_error=True, **kw):
        """Refine the columns of X in place (eigref_refine_dense)."""
        pa, n, lda, ka = _dense_a(A)
        px, nx, k, ldx, kx = _colmajor(X)
        if nx != n:
            raise ValueError("X has %d rows, A is %d x %d" % (nx, n, n))
        p = self.params(**kw)
        rep, want = self._report(k, p.max_iters, history)
        st = lib().eigref_refine_dense(self._h, pa, n, lda, px, ldx, k, ctypes.byref(p), ctypes.byref(rep))
        return self._finish(st, rep, k, want, raise_on_error)

    def refine_csr(self, row_ptr, col_idx, val, X, history=False, raise_on_error=True, **kw):
        """Refine the columns of X in place against a CSR matrix (eigref_refine_csr)."""
        prp, n1, k1 = _int32(row_ptr, "row_ptr")
        pci, nnz, k2 = _int32(col_idx, "col_idx")
        pv, nnz2, k3 = _f64vec(val, "val")
        px, n, k, ldx, kx = _colmajor(X)
        if n1 != n + 1 or nnz2 != nnz:
            raise ValueError("inconsistent CSR sizes")
        p = self.params(**kw)
        rep, want = self._report(k, p.max_iters, history)
        st = lib().eigref_refine_csr(self._h, prp, pci, pv, n, nnz, px, ldx, k, ctypes.byref(p), ctypes.byref(rep))
        return self._finish(st, rep, k, want, raise_on_error)

    def refine_batched(self, problems, history=False, raise_on_error=True, **kw):
        """Refine many dense problems at once (eigref_refine_batched).

        problems: sequence of dicts with keys A, X (device tensors, X
        column-major, refined in place) and optionally target, shift, norm_a.
        kw: the shared options.  Returns (status, list of per-problem reports)."""
        count = len(problems)
        arr = (Problem * count)()
        keep, wants, reps = [], [], (Report * count)()
        p = self.params(**kw)
        for i, pb in enumerate(problems):
            pa, n, lda, ka = _dense_a(pb["A"])
            px, nx, k, ldx, kx = _colmajor(pb["X"])
            if nx != n:
                raise ValueError("problem %d: X has %d rows, A is %d x %d" % (i, nx, n, n))
            t = pb.get("target", "largest_mag")
            arr[i] = Problem(pa, n, lda, px, ldx, k, TARGETS[t] if isinstance(t, str) else int(t),
                             float(pb.get("shift", 0.0)), float(pb.get("norm_a", 0.0)))
            rep, want = self._report(k, p.max_iters, history)
            reps[i] = rep
            keep.append((ka, kx))
            wants.append((k, want))
        st = lib().eigref_refine_batched(self._h, count, arr, ctypes.byref(p), reps)
        outs = [self._finish(reps[i].status, reps[i], k, want, False) for i, (k, want) in enumerate(wants)]
        if raise_on_error and st in (E_INVALID, E_CUDA, E_NOMEM, E_UNSUPPORTED):
            raise EigrefError(st, self.last_error())
        return st, outs

    def gram(self, X, P, G, S, precision="fp64", slices=0):
        """G = X^T X, S = X^T P (eigref_gram); X, P column-major device arrays,
        G, S k x k column-major, written in place."""
        px, n, k, ldx, kx = _colmajor(X)
        pp, n2, k2, ldp, kp = _colmajor(P, "P")
        pg, ng, kg_, _, kg = _colmajor(G, "G")
        ps, ns, ks_, _, ks = _colmajor(S, "S")
        _same_shape("P", (n2, k2), (n, k))
        _same_shape("G", (ng, kg_), (k, k))
        _same_shape("S", (ns, ks_), (k, k))
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        st = lib().eigref_gram(self._h, px, ldx, pp, ldp, n, k, prec, int(slices), pg, ps)
        if st != OK:
            raise EigrefError(st, self.last_error())

    def product_dense(self, A, X, P, shift=0.0, precision="fp64", slices=0):
        """P = (A - shift I) X (eigref_product_dense); P column-major, written in place."""
        pa, n, lda, ka = _dense_a(A)
        px, nx, k, ldx, kx = _colmajor(X)
        pp, np_, kp, ldp, kpp = _colmajor(P, "P")
        _same_shape("X", (nx, k), (n, k))
        _same_shape("P", (np_, kp), (n, k))
        prec = PRECISIONS[precision] if isinstance(precision, str) else precision
        st = lib().eigref_product_dense(self._h, pa, n, lda, px, ldx, k, float(shift), prec, int(slices), pp, ldp)
        if st != OK:
            raise EigrefError(st, self.last_error())

    def product_csr(self, row_ptr, col_idx, val, X, P, shift=0.0):
        """P = (A - shift I) X for CSR A (eigref_product_csr)."""
        prp, n1, k1 = _int32(row_ptr, "row_ptr")
        pci, nnz, k2 = _int32(col_idx, "col_idx")
        pv, nnz2, k3 = _f64vec(val, "val")
        px, n, k, ldx, kx = _colmajor(X)
        pp, np_, kp, ldp, kpp = _colmajor(P, "P")
        if n1 != n + 1 or nnz2 != nnz:
            raise ValueError("inconsistent CSR sizes")
        _same_shape("P", (np_, kp), (n, k))
        st = lib().eigref_product_csr(self._h, prp, pci, pv, n, nnz, px, ldx, k, float(shift), pp, ldp)
        if st != OK:
            raise EigrefError(st, self.last_error())
