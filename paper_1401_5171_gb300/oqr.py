"""Python binding of liboqr (include/oqr.h): argument marshalling only.

The C entry points are exposed under their own names (``oqr_cholqr``,
``oqr_cholqr2``, ``oqr_cgs2``, ...) and take raw device pointers and leading
dimensions, exactly as declared in the header.  ``Oqr`` wraps a context and
accepts torch tensors: a matrix argument is a 2-D float64 CUDA tensor stored
column-major (``x.stride(0) == 1``; leading dimension ``x.stride(1)``), which
``colmajor`` produces from any tensor.  Every computation runs in the CUDA
library; if it cannot be loaded this module raises, it never falls back.
"""
from __future__ import annotations

import ctypes
import os
import re

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liboqr.so")
HEADERS = [os.path.join(os.path.dirname(HERE), "include", "oqr.h")]

OQR_OK, OQR_ERR_INVALID_ARG, OQR_ERR_NOT_SPD, OQR_ERR_CHECK_FAILED = 0, 1, 2, 3
OQR_ERR_CUDA, OQR_ERR_NO_MEMORY, OQR_ERR_TIMEOUT, OQR_ERR_UNSUPPORTED = 4, 5, 6, 7
OQR_FP64, OQR_BF16X3, OQR_FP8, OQR_FP64_TC, OQR_TC2 = 0, 1, 2, 3, 4
OQR_BATCH_CHOLQR_TC, OQR_BATCH_CHOLQR2_TC2, OQR_BATCH_CHOLQR2_TC, OQR_BATCH_SCHOLQR3_TC = 0, 1, 2, 3
OQR_ALGO_CHOLQR, OQR_ALGO_CHOLQR2, OQR_ALGO_SCHOLQR3, OQR_ALGO_CGS2 = 0, 1, 2, 3
OQR_BATCHED_FP64, OQR_BATCHED_TC, OQR_BATCHED_TC2_FIRST, OQR_BATCHED_SHIFTED_TC, OQR_BATCHED_SELECTOR = 0, 1, 2, 3, 4


class oqr_opts(ctypes.Structure):
    _fields_ = [("passes", ctypes.c_int), ("shifted", ctypes.c_int), ("prec", ctypes.c_int),
                ("shift_c", ctypes.c_double), ("block", ctypes.c_int), ("check", ctypes.c_int),
                ("spin_limit", ctypes.c_long), ("final_prec", ctypes.c_int), ("prec_mid", ctypes.c_int),
                ("reuse_w", ctypes.c_int), ("batch_splits", ctypes.c_void_p), ("selector_params", ctypes.c_void_p),
                ("selector_tol", ctypes.c_double), ("selector_check", ctypes.c_int), ("batch_orth", ctypes.c_void_p),
                ("batch_choice", ctypes.c_void_p)]


class oqr_info(ctypes.Structure):
    _fields_ = [("info", ctypes.c_int), ("passes_run", ctypes.c_int), ("orth_err", ctypes.c_double),
                ("shift", ctypes.c_double)]


class OqrError(RuntimeError):
    def __init__(self, status, what, info=0):
        self.status = status
        self.info = info
        super().__init__(f"{what}: {status_string(status)} (info={info})")


_lib = None


def declared_functions(headers=None):
    """Names of the functions declared in include/*.h (used by the export test)."""
    names = []
    for h in headers or HEADERS:
        txt = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*(oqr_[a-z0-9_]+)\s*\(", txt, flags=re.M)
    return sorted(set(names))


def load(path: str | None = None):
    """Loads liboqr.so (building it first if it is missing and nvcc is present)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        from . import build as _build
        _build.build()
    if not os.path.exists(p):
        raise RuntimeError(f"liboqr.so not found at {p}: build it with paper_1401_5171_gb300/build.py")
    lib = ctypes.CDLL(p)
    vp, i, l, d = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    S = ctypes.c_int
    po, pi = ctypes.POINTER(oqr_opts), ctypes.POINTER(oqr_info)
    lib.oqr_default_opts.argtypes = [po]
    lib.oqr_default_opts.restype = None
    lib.oqr_status_string.argtypes = [S]
    lib.oqr_status_string.restype = ctypes.c_char_p
    lib.oqr_create.argtypes = [ctypes.POINTER(vp), i]
    lib.oqr_destroy.argtypes = [vp]
    lib.oqr_workspace_size.argtypes = [vp, i, i, i, po, ctypes.POINTER(ctypes.c_size_t)]
    lib.oqr_set_workspace.argtypes = [vp, vp, ctypes.c_size_t]
    lib.oqr_get_status.argtypes = [vp, vp, ctypes.POINTER(i)]
    qr = [vp, i, i, vp, l, vp, l, vp, l, vp, l, po, pi, vp]
    for name in ("oqr_cholqr", "oqr_cholqr2", "oqr_cgs2"):
        getattr(lib, name).argtypes = qr
    lib.oqr_gram.argtypes = [vp, i, i, vp, l, vp, l, vp, l, i, vp]
    lib.oqr_gram_noalloc.argtypes = [i, i, vp, l, vp, l, vp, l, vp]
    pl = ctypes.POINTER(ctypes.c_long)
    ppd = ctypes.POINTER(ctypes.c_void_p)
    lib.oqr_batched.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ppd, pl, ppd, pl, ppd, pl, ppd, pl, i,
                                po, vp, vp]
    lib.oqr_batched_features.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ppd, pl, ppd, pl, vp, vp]
    lib.oqr_batched_mixed.argtypes = [vp, i, ctypes.POINTER(i), ctypes.POINTER(i), ppd, pl, ppd, pl, ppd, pl, ppd,
                                      pl, ctypes.POINTER(i), vp, vp, vp]
    lib.oqr_batched_default_splits.argtypes = [i, i]
    fp, ip = ctypes.c_void_p, ctypes.c_void_p
    lib.oqr_features.argtypes = [vp, i, i, vp, l, vp, l, fp, vp]
    lib.oqr_mlp_param_count.argtypes = []
    lib.oqr_mlp_forward.argtypes = [vp, i, fp, fp, i, fp, ip, vp]
    lib.oqr_mlp_grad.argtypes = [vp, i, fp, ip, fp, fp, fp, vp]
    lib.oqr_mlp_adam.argtypes = [vp, fp, fp, fp, fp, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                                 ctypes.c_float, i, vp]
    lib.oqr_gram_phases.argtypes = [vp, i, i, vp, l, vp, l, vp, l, i, ctypes.POINTER(ctypes.c_float),
                                    ctypes.POINTER(i), vp]
    lib.oqr_potrf.argtypes = [vp, i, vp, l, d, vp, l, ctypes.POINTER(i), vp]
    lib.oqr_trsm.argtypes = [vp, i, i, vp, l, vp, l, vp, l, vp]
    lib.oqr_trsm_tc.argtypes = [vp, i, i, vp, l, vp, l, vp, l, vp]
    lib.oqr_trsm_last.argtypes = [vp, i, i, vp, l, vp, l, vp, l, vp, l, vp]
    lib.oqr_cholqr2_host.argtypes = [vp, i, i, vp, l, vp, l, vp, l, vp, l, po, pi, vp]
    lib.oqr_rprod.argtypes = [vp, i, vp, l, vp, l, vp, l, vp]
    lib.oqr_check.argtypes = [vp, i, i, vp, l, vp, l, vp, l, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    lib.oqr_repres.argtypes = [vp, i, i, vp, l, vp, l, vp, l, ctypes.POINTER(d), ctypes.POINTER(d), vp]
    lib.oqr_diag_timeout.argtypes = [vp, l, vp]
    lib.oqr_set_batch_budget.argtypes = [vp, ctypes.c_size_t]
    lib.oqr_glls.argtypes = [vp, i, i, i, vp, l, vp, l, vp, l, vp, l, vp, l, vp]
    lib.oqr_cholqr2_tridiag.argtypes = [vp, i, i, vp, vp, vp, l, vp, l, vp, l, po, pi, vp]
    lib.oqr_precholqr.argtypes = qr
    lib.oqr_precholqr_tridiag.argtypes = [vp, i, i, vp, vp, vp, l, vp, l, vp, l, po, pi, vp]
    lib.oqr_tsqr.argtypes = [vp, i, i, vp, l, vp, l, vp, l, vp]
    lib.oqr_gram_tridiag.argtypes = [vp, i, i, vp, vp, vp, l, vp, l, i, vp]
    lib.oqr_symm.argtypes = [vp, i, i, vp, l, vp, l, vp, l, vp]
    for name in declared_functions():
        f = getattr(lib, name)
        if f.restype is ctypes.c_int or name not in ("oqr_default_opts", "oqr_status_string"):
            if name not in ("oqr_default_opts", "oqr_status_string"):
                f.restype = S
    _lib = lib
    return lib


def status_string(s: int) -> str:
    return load().oqr_status_string(int(s)).decode()


# ---- raw entry points, same names as the C ABI ------------------------------
def _raw(name):
    def f(*args):
        return getattr(load(), name)(*args)
    f.__name__ = name
    return f


for _n in ("oqr_default_opts", "oqr_create", "oqr_destroy", "oqr_workspace_size", "oqr_set_workspace",
           "oqr_get_status", "oqr_cholqr", "oqr_cholqr2", "oqr_cholqr2_host", "oqr_cgs2", "oqr_gram", "oqr_gram_noalloc", "oqr_gram_phases", "oqr_potrf", "oqr_trsm", "oqr_trsm_tc", "oqr_trsm_last",
           "oqr_rprod", "oqr_check", "oqr_repres", "oqr_diag_timeout", "oqr_set_batch_budget", "oqr_batched", "oqr_batched_mixed", "oqr_batched_default_splits", "oqr_features",
           "oqr_mlp_param_count", "oqr_mlp_forward", "oqr_mlp_grad", "oqr_mlp_adam", "oqr_glls", "oqr_symm", "oqr_cholqr2_tridiag", "oqr_gram_tridiag",
           "oqr_precholqr", "oqr_precholqr_tridiag", "oqr_tsqr", "oqr_batched_features"):
    globals()[_n] = _raw(_n)


# ---- tensor-level convenience -------------------------------------------------
def _leading_dim(x):
    """Leading dimension of a column-major 2-D tensor, or None if it is not column-major.

    Strides of size-1 dimensions carry no information (torch normalises them),
    so a single column has leading dimension = its row count and a single row
    needs no unit row stride.
    """
    rows, cols = x.shape
    if rows > 1 and x.stride(0) != 1:
        return None
    ld = x.stride(1) if cols > 1 else rows
    return ld if ld >= max(1, rows) else None


def colmajor(x):
    """Column-major copy (or view) of a 2-D tensor: element (i, j) at i + j * ld."""
    if x.dim() == 1:
        x = x.reshape(-1, 1)
    if _leading_dim(x) is not None:
        return x
    return x.t().contiguous().t()


def _m(x, host=False):
    if x.dtype.is_floating_point is False or x.element_size() != 8:
        raise TypeError("liboqr matrices are float64")
    if x.is_cuda == host:
        raise TypeError("this call takes host matrices" if host else "liboqr matrices live in device memory")
    ld = _leading_dim(x) if x.dim() == 2 else None
    if ld is None:
        raise ValueError("matrix must be 2-D column-major (stride(0) == 1); use colmajor()")
    return ctypes.c_void_p(x.data_ptr()), ctypes.c_long(max(1, ld))


def _vec(x, length):
    """Device pointer of a contiguous 1-D float64 CUDA tensor of at least `length` entries (None if length 0)."""
    if length <= 0:
        return None if x is None else ctypes.c_void_p(x.data_ptr())
    if x is None or x.dim() != 1 or x.dtype.itemsize != 8 or not x.is_cuda or x.stride(0) != 1 or x.numel() < length:
        raise ValueError("expected a contiguous 1-D float64 CUDA tensor")
    return ctypes.c_void_p(x.data_ptr())


def empty_colmajor(rows, cols, device, dtype=None):
    import torch
    return torch.empty((cols, rows), dtype=dtype or torch.float64, device=device).t()


def make_opts(**kw) -> oqr_opts:
    o = oqr_opts()
    load().oqr_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


class Oqr:
    """A liboqr context on one device; methods take column-major float64 CUDA tensors."""

    def __init__(self, device: int = 0):
        self.lib = load()
        self.device = device
        self.ctx = ctypes.c_void_p()
        st = self.lib.oqr_create(ctypes.byref(self.ctx), int(device))
        if st != OQR_OK:
            raise OqrError(st, "oqr_create")

    def close(self):
        if self.ctx:
            self.lib.oqr_destroy(self.ctx)
            self.ctx = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @staticmethod
    def _stream(stream):
        import torch
        s = stream if stream is not None else torch.cuda.current_stream()
        return ctypes.c_void_p(s.cuda_stream)

    def _qr(self, name, A, Z, Q=None, R=None, opts=None, stream=None, sync=True, raise_on_error=True, **kw):
        m, n = Z.shape
        Q = Q if Q is not None else empty_colmajor(m, n, Z.device)
        R = R if R is not None else empty_colmajor(n, n, Z.device)
        o = opts if opts is not None else make_opts(**kw)
        info = oqr_info()
        a, lda = _m(A)
        z, ldz = _m(Z)
        q, ldq = _m(Q)
        r, ldr = _m(R)
        st = getattr(self.lib, name)(self.ctx, m, n, a, lda, z, ldz, q, ldq, r, ldr, ctypes.byref(o),
                                     ctypes.byref(info) if sync else None, self._stream(stream))
        if st != OQR_OK and raise_on_error:
            raise OqrError(st, name, info.info)
        return Q, R, (st, info)

    def oqr_cholqr(self, A, Z, **kw):
        return self._qr("oqr_cholqr", A, Z, **kw)

    def oqr_cholqr2(self, A, Z, **kw):
        return self._qr("oqr_cholqr2", A, Z, **kw)

    def oqr_cholqr2_host(self, A, Z, Q=None, R=None, opts=None, stream=None, sync=True, raise_on_error=True, **kw):
        """oqr_cholqr2 on host (CPU, preferably pinned) column-major tensors; returns (Q, R, (status, info))."""
        import torch
        m, n = Z.shape
        Q = Q if Q is not None else torch.empty((n, m), dtype=torch.float64, pin_memory=True).t()
        R = R if R is not None else torch.empty((n, n), dtype=torch.float64, pin_memory=True).t()
        o = opts if opts is not None else make_opts(**kw)
        info = oqr_info()
        a, lda = _m(A, host=True)
        z, ldz = _m(Z, host=True)
        q, ldq = _m(Q, host=True)
        r, ldr = _m(R, host=True)
        st = self.lib.oqr_cholqr2_host(self.ctx, m, n, a, lda, z, ldz, q, ldq, r, ldr, ctypes.byref(o),
                                       ctypes.byref(info) if sync else None, self._stream(stream))
        if st != OQR_OK and raise_on_error:
            raise OqrError(st, "oqr_cholqr2_host", info.info)
        return Q, R, (st, info)

    def oqr_cgs2(self, A, Z, **kw):
        return self._qr("oqr_cgs2", A, Z, **kw)

    def oqr_gram(self, A, Z, G=None, prec=OQR_FP64, stream=None):
        n = Z.shape[1]
        G = G if G is not None else empty_colmajor(n, n, Z.device)
        a, lda = _m(A)
        z, ldz = _m(Z)
        g, ldg = _m(G)
        st = self.lib.oqr_gram(self.ctx, Z.shape[0], n, a, lda, z, ldz, g, ldg, prec, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_gram")
        return G

    def oqr_gram_phases(self, A, Z, prec, G=None, stream=None):
        """Per-phase CUDA-event times (ms) of the Gram pipeline; see include/oqr.h."""
        n = Z.shape[1]
        G = G if G is not None else empty_colmajor(n, n, Z.device)
        a, lda = _m(A)
        z, ldz = _m(Z)
        g, ldg = _m(G)
        ms = (ctypes.c_float * 8)()
        k = ctypes.c_int(0)
        st = self.lib.oqr_gram_phases(self.ctx, Z.shape[0], n, a, lda, z, ldz, g, ldg, prec, ms, ctypes.byref(k),
                                      self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_gram_phases")
        return [ms[i] for i in range(k.value)], G

    def _batch_args(self, As, Zs, Qs, Rs, status):
        import torch
        cnt = len(Zs)
        if len(As) != cnt or (Qs is not None and len(Qs) != cnt) or (Rs is not None and len(Rs) != cnt):
            raise ValueError("As, Zs, Qs and Rs need one entry per instance")
        Qs = Qs if Qs is not None else [empty_colmajor(z.shape[0], z.shape[1], z.device) for z in Zs]
        Rs = Rs if Rs is not None else [empty_colmajor(z.shape[1], z.shape[1], z.device) for z in Zs]
        I = ctypes.c_int * cnt
        L = ctypes.c_long * cnt
        P = ctypes.c_void_p * cnt
        mm = I(*[z.shape[0] for z in Zs])
        nn = I(*[z.shape[1] for z in Zs])
        ap, al, zp, zl, qp, ql, rp, rl = P(), L(), P(), L(), P(), L(), P(), L()
        for b in range(cnt):
            (ap[b], al[b]), (zp[b], zl[b]) = _m(As[b]), _m(Zs[b])
            (qp[b], ql[b]), (rp[b], rl[b]) = _m(Qs[b]), _m(Rs[b])
        st = status if status is not None else torch.empty(cnt, dtype=torch.int32, device=Zs[0].device)
        return Qs, Rs, st, (cnt, mm, nn, ap, al, zp, zl, qp, ql, rp, rl)

    def oqr_batched(self, As, Zs, Qs=None, Rs=None, splits=None, stream=None, status=None, mode=0, params=None,
                    tol=1e-12, check_all=False, orth=None, choice=None):
        """Batched oblique QR over lists of column-major CUDA tensors; returns (Qs, Rs, status tensor).

        mode: OQR_BATCHED_FP64 (splits: the work plan), OQR_BATCHED_TC, OQR_BATCHED_TC2_FIRST,
        OQR_BATCHED_SHIFTED_TC, or OQR_BATCHED_SELECTOR (params: the trained network, a float32 CUDA tensor;
        tol, check_all: the selector's check).  orth (float64) and choice (int32) CUDA tensors of one entry
        per instance, when given, receive the checks and (selector) the options used."""
        Qs, Rs, st, a = self._batch_args(As, Zs, Qs, Rs, status)
        if splits is not None and len(splits) != a[0]:
            raise ValueError("splits needs one entry per instance")
        sp = (ctypes.c_int * a[0])(*splits) if splits is not None else None
        o = make_opts()
        o.batch_splits = ctypes.cast(sp, ctypes.c_void_p) if sp is not None else None
        o.selector_params = params.data_ptr() if params is not None else None
        o.selector_tol = float(tol)
        o.selector_check = 1 if check_all else 0
        o.batch_orth = orth.data_ptr() if orth is not None else None
        o.batch_choice = choice.data_ptr() if choice is not None else None
        r = self.lib.oqr_batched(self.ctx, *a, int(mode), ctypes.byref(o), ctypes.c_void_p(st.data_ptr()),
                                 self._stream(stream))
        if r != OQR_OK:
            raise OqrError(r, "oqr_batched")
        return Qs, Rs, st

    def oqr_batched_features(self, As, Zs, stream=None):
        """The selector's features (count x 16 float32 CUDA tensor) after each instance's first FP64-accurate
        pass."""
        import torch
        cnt = len(Zs)
        I = ctypes.c_int * cnt
        L = ctypes.c_long * cnt
        P = ctypes.c_void_p * cnt
        mm = I(*[z.shape[0] for z in Zs])
        nn = I(*[z.shape[1] for z in Zs])
        ap, al, zp, zl = P(), L(), P(), L()
        for b in range(cnt):
            (ap[b], al[b]), (zp[b], zl[b]) = _m(As[b]), _m(Zs[b])
        feat = torch.empty((cnt, 16), dtype=torch.float32, device=Zs[0].device)
        r = self.lib.oqr_batched_features(self.ctx, cnt, mm, nn, ap, al, zp, zl, ctypes.c_void_p(feat.data_ptr()),
                                          self._stream(stream))
        if r != OQR_OK:
            raise OqrError(r, "oqr_batched_features")
        return feat

    def oqr_batched_mixed(self, As, Zs, program=None, Qs=None, Rs=None, stream=None, status=None, check=False):
        """Batched oblique QR on the tensor cores; program: per-instance OQR_BATCH_* (None: all
        OQR_BATCH_CHOLQR2_TC).  Returns (Qs, Rs, status tensor), and with check=True also the tensor of
        per-instance ||Q^T A Q - I||_2 estimates."""
        import torch
        Qs, Rs, st, a = self._batch_args(As, Zs, Qs, Rs, status)
        if program is not None and len(program) != a[0]:
            raise ValueError("program needs one entry per instance")
        pr = (ctypes.c_int * a[0])(*[int(x) for x in program]) if program is not None else None
        orth = torch.empty(a[0], dtype=torch.float64, device=Zs[0].device) if check else None
        r = self.lib.oqr_batched_mixed(self.ctx, *a, pr, ctypes.c_void_p(st.data_ptr()),
                                       ctypes.c_void_p(orth.data_ptr()) if check else None, self._stream(stream))
        if r != OQR_OK:
            raise OqrError(r, "oqr_batched_mixed")
        return (Qs, Rs, st, orth) if check else (Qs, Rs, st)

    # ---- selector ---------------------------------------------------------------
    def oqr_features(self, A, Z, out=None, stream=None):
        import torch
        f = out if out is not None else torch.empty(16, dtype=torch.float32, device=Z.device)
        a, lda = _m(A)
        z, ldz = _m(Z)
        st = self.lib.oqr_features(self.ctx, Z.shape[0], Z.shape[1], a, lda, z, ldz, ctypes.c_void_p(f.data_ptr()),
                                   self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_features")
        return f

    def oqr_mlp_forward(self, X, params, bf16=True, stream=None, want_logits=True):
        import torch
        B = X.shape[0]
        logits = torch.empty((B, 4), dtype=torch.float32, device=X.device) if want_logits else None
        choice = torch.empty(B, dtype=torch.int32, device=X.device)
        st = self.lib.oqr_mlp_forward(self.ctx, B, ctypes.c_void_p(X.contiguous().data_ptr()),
                                      ctypes.c_void_p(params.data_ptr()), int(bf16),
                                      ctypes.c_void_p(logits.data_ptr()) if logits is not None else None,
                                      ctypes.c_void_p(choice.data_ptr()), self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_mlp_forward")
        return logits, choice

    def oqr_mlp_grad(self, X, y, params, stream=None):
        import torch
        grad = torch.empty_like(params)
        loss = torch.empty(1, dtype=torch.float32, device=X.device)
        st = self.lib.oqr_mlp_grad(self.ctx, X.shape[0], ctypes.c_void_p(X.contiguous().data_ptr()),
                                   ctypes.c_void_p(y.data_ptr()), ctypes.c_void_p(params.data_ptr()),
                                   ctypes.c_void_p(grad.data_ptr()), ctypes.c_void_p(loss.data_ptr()),
                                   self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_mlp_grad")
        return grad, loss

    def oqr_mlp_adam(self, params, grad, m, v, lr, t, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        st = self.lib.oqr_mlp_adam(self.ctx, ctypes.c_void_p(params.data_ptr()), ctypes.c_void_p(grad.data_ptr()),
                                   ctypes.c_void_p(m.data_ptr()), ctypes.c_void_p(v.data_ptr()), lr, beta1, beta2,
                                   eps, int(t), self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_mlp_adam")

    def oqr_potrf(self, G, shift=0.0, R=None, stream=None):
        n = G.shape[0]
        R = R if R is not None else empty_colmajor(n, n, G.device)
        g, ldg = _m(G)
        r, ldr = _m(R)
        info = ctypes.c_int(0)
        st = self.lib.oqr_potrf(self.ctx, n, g, ldg, float(shift), r, ldr, ctypes.byref(info), self._stream(stream))
        return R, st, info.value

    def oqr_trsm(self, Z, R, Q=None, stream=None, name="oqr_trsm"):
        m, n = Z.shape
        Q = Q if Q is not None else empty_colmajor(m, n, Z.device)
        z, ldz = _m(Z)
        r, ldr = _m(R)
        q, ldq = _m(Q)
        st = getattr(self.lib, name)(self.ctx, m, n, z, ldz, r, ldr, q, ldq, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, name)
        return Q

    def oqr_trsm_tc(self, Z, R, Q=None, stream=None):
        return self.oqr_trsm(Z, R, Q=Q, stream=stream, name="oqr_trsm_tc")

    def oqr_trsm_last(self, G, Z, R, Q=None, stream=None):
        m, n = Z.shape
        Q = Q if Q is not None else empty_colmajor(m, n, Z.device)
        g, ldg = _m(G)
        z, ldz = _m(Z)
        r, ldr = _m(R)
        q, ldq = _m(Q)
        st = self.lib.oqr_trsm_last(self.ctx, m, n, g, ldg, z, ldz, r, ldr, q, ldq, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_trsm_last")
        return Q

    def oqr_rprod(self, U, S, R=None, stream=None):
        n = U.shape[0]
        R = R if R is not None else empty_colmajor(n, n, U.device)
        u, ldu = _m(U)
        s_, lds = _m(S)
        r, ldr = _m(R)
        st = self.lib.oqr_rprod(self.ctx, n, u, ldu, s_, lds, r, ldr, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_rprod")
        return R

    def oqr_check(self, A, Q, want_E=False, stream=None):
        m, n = Q.shape
        E = empty_colmajor(n, n, Q.device) if want_E else None
        a, lda = _m(A)
        q, ldq = _m(Q)
        e, lde = _m(E) if E is not None else (None, ctypes.c_long(n))
        o2, of = ctypes.c_double(), ctypes.c_double()
        st = self.lib.oqr_check(self.ctx, m, n, a, lda, q, ldq, e, lde, ctypes.byref(o2), ctypes.byref(of),
                                self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_check")
        return o2.value, of.value, E

    def oqr_diag_timeout(self, limit_ns, stream=None):
        """One device-side wait that nothing completes; returns the context's status afterwards."""
        st = self.lib.oqr_diag_timeout(self.ctx, int(limit_ns), self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_diag_timeout")
        return self.status(stream)

    def status(self, stream=None):
        """The context's device-side status (synchronizes the stream)."""
        info = ctypes.c_int(0)
        return self.lib.oqr_get_status(self.ctx, self._stream(stream), ctypes.byref(info))

    def set_batch_budget(self, nbytes):
        """Slice-plane bytes per wave of the tensor-core batches (0: the default)."""
        st = self.lib.oqr_set_batch_budget(self.ctx, int(nbytes))
        if st != OQR_OK:
            raise OqrError(st, "oqr_set_batch_budget")

    def set_workspace(self, ptr, nbytes):
        """Hands the context a caller-owned device buffer (ptr = 0: the context allocates again)."""
        st = self.lib.oqr_set_workspace(self.ctx, ctypes.c_void_p(ptr) if ptr else None, int(nbytes))
        if st != OQR_OK:
            raise OqrError(st, "oqr_set_workspace")

    def oqr_precholqr(self, A, Z, **kw):
        return self._qr("oqr_precholqr", A, Z, **kw)

    def oqr_precholqr_tridiag(self, d, e, Z, **kw):
        return self.oqr_cholqr2_tridiag(d, e, Z, _name="oqr_precholqr_tridiag", **kw)

    def oqr_tsqr(self, Z, Y=None, S=None, stream=None):
        """Euclidean Householder QR Z = Y S (S upper triangular with a positive diagonal)."""
        m, n = Z.shape
        Y = Y if Y is not None else empty_colmajor(m, n, Z.device)
        S = S if S is not None else empty_colmajor(n, n, Z.device)
        z, ldz = _m(Z)
        y, ldy = _m(Y)
        s_, lds = _m(S)
        st = self.lib.oqr_tsqr(self.ctx, m, n, z, ldz, y, ldy, s_, lds, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_tsqr")
        return Y, S

    def oqr_cholqr2_tridiag(self, d, e, Z, Q=None, R=None, opts=None, stream=None, sync=True, raise_on_error=True,
                            _name="oqr_cholqr2_tridiag", **kw):
        """The normal-equation method for tridiagonal A (diagonal d, off-diagonal e: 1-D float64 CUDA tensors);
        returns (Q, R, (status, info))."""
        m, n = Z.shape
        Q = Q if Q is not None else empty_colmajor(m, n, Z.device)
        R = R if R is not None else empty_colmajor(n, n, Z.device)
        o = opts if opts is not None else make_opts(**kw)
        info = oqr_info()
        z, ldz = _m(Z)
        q, ldq = _m(Q)
        r, ldr = _m(R)
        st = getattr(self.lib, _name)(self.ctx, m, n, _vec(d, m), _vec(e, m - 1), z, ldz, q, ldq, r, ldr,
                                      ctypes.byref(o), ctypes.byref(info) if sync else None, self._stream(stream))
        if st != OQR_OK and raise_on_error:
            raise OqrError(st, _name, info.info)
        return Q, R, (st, info)

    def oqr_gram_tridiag(self, d, e, Z, G=None, prec=OQR_FP64, stream=None):
        m, n = Z.shape
        G = G if G is not None else empty_colmajor(n, n, Z.device)
        z, ldz = _m(Z)
        g, ldg = _m(G)
        st = self.lib.oqr_gram_tridiag(self.ctx, m, n, _vec(d, m), _vec(e, m - 1), z, ldz, g, ldg, prec,
                                       self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_gram_tridiag")
        return G

    def oqr_symm(self, A, B, C=None, stream=None):
        """C = A B for symmetric A (lower triangle read)."""
        m, k = B.shape
        C = C if C is not None else empty_colmajor(m, k, B.device)
        a, lda = _m(A)
        b, ldb = _m(B)
        c, ldc = _m(C)
        st = self.lib.oqr_symm(self.ctx, m, k, a, lda, b, ldb, c, ldc, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_symm")
        return C

    def oqr_glls(self, A, Q, R, B, X=None, stream=None):
        """x = R^{-1} Q^T A b for each column b of B (Sec. 1's generalized least squares)."""
        m, n = Q.shape
        k = B.shape[1]
        X = X if X is not None else empty_colmajor(n, k, B.device)
        a, lda = _m(A)
        q, ldq = _m(Q)
        r, ldr = _m(R)
        b, ldb = _m(B)
        x, ldx = _m(X)
        st = self.lib.oqr_glls(self.ctx, m, n, k, a, lda, q, ldq, r, ldr, b, ldb, x, ldx, self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_glls")
        return X

    def oqr_repres(self, Z, Q, R, stream=None):
        """(||Z - Q R||_2 / ||Z||_2 estimate, ||Z - Q R||_F / ||Z||_F)."""
        m, n = Z.shape
        z, ldz = _m(Z)
        q, ldq = _m(Q)
        r, ldr = _m(R)
        r2, rf = ctypes.c_double(), ctypes.c_double()
        st = self.lib.oqr_repres(self.ctx, m, n, z, ldz, q, ldq, r, ldr, ctypes.byref(r2), ctypes.byref(rf),
                                 self._stream(stream))
        if st != OQR_OK:
            raise OqrError(st, "oqr_repres")
        return r2.value, rf.value
