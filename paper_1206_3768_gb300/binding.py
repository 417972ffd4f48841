"""Thin ctypes binding of the C ABI in include/chfsi.h (argument marshalling only).

Every function here has the name of the C entry point it calls.  Matrices are torch
complex128 tensors in natural (row, column) indexing; they are handed to the library in
column-major storage (``fortran`` makes a column-major copy only when needed).  Device
tensors are passed as device pointers, CPU tensors as host pointers (the solve entry
points accept both; the step entry points need CUDA tensors).

The library is the in-tree ``_lib/libchfsi.so`` built by ``build.py``; if it is missing
or cannot be loaded, every call raises: there is no fallback implementation.

Every context created here runs on torch's current CUDA stream (unless a stream is passed),
so tensors produced by torch just before a call are complete when the library reads them.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, c_char, c_char_p, c_double, c_int32, c_int64, c_uint64, c_void_p

import torch

from . import build as _build

CHFSI_OK, CHFSI_EINVAL, CHFSI_ENOTPD, CHFSI_ENOCONV, CHFSI_ECUDA, CHFSI_ETIMEOUT, CHFSI_ENOMEM = range(7)
_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOTPD", 3: "ENOCONV", 4: "ECUDA", 5: "ETIMEOUT", 6: "ENOMEM"}


class ChfsiError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"CHFSI_{_NAMES.get(code, code)}: {msg}")
        self.code = code


MLP_IN, MLP_HID = 8, 64
MLP_SIZES = (MLP_IN, MLP_HID, MLP_HID, MLP_HID, 1)
MLP_NPARAM = MLP_HID * MLP_IN + MLP_HID + 2 * (MLP_HID * MLP_HID + MLP_HID) + MLP_HID + 1  # 8961
DEGREE_LOG_FIELDS = 20


class chfsi_mlp(ctypes.Structure):
    _fields_ = [("w1", ctypes.c_float * (MLP_HID * MLP_IN)), ("b1", ctypes.c_float * MLP_HID),
                ("w2", ctypes.c_float * (MLP_HID * MLP_HID)), ("b2", ctypes.c_float * MLP_HID),
                ("w3", ctypes.c_float * (MLP_HID * MLP_HID)), ("b3", ctypes.c_float * MLP_HID),
                ("w4", ctypes.c_float * MLP_HID), ("b4", ctypes.c_float),
                ("mean", ctypes.c_float * MLP_IN), ("scale", ctypes.c_float * MLP_IN)]

    def params(self):
        """The MLP_NPARAM trainable parameters in the order w1, b1, .., w4, b4 (numpy copy)."""
        import numpy as np

        return np.ctypeslib.as_array((ctypes.c_float * MLP_NPARAM).from_address(ctypes.addressof(self))).copy()

    def set_params(self, p):
        """Overwrite the trainable parameters from a flat array in the order of params()."""
        import numpy as np

        a = np.ascontiguousarray(np.asarray(p, dtype=np.float32))
        if a.size != MLP_NPARAM:
            raise ValueError("need MLP_NPARAM parameters")
        ctypes.memmove(ctypes.addressof(self), a.ctypes.data, 4 * MLP_NPARAM)


class chfsi_opts(ctypes.Structure):
    _fields_ = [("deg_min", c_int32), ("deg_max", c_int32), ("max_loops", c_int32),
                ("lanczos_k_warm", c_int32), ("lanczos_k_cold", c_int32),
                ("reuse_factor", c_int32), ("precision", c_int32), ("slices_max", c_int32),
                ("seed", c_uint64), ("cuda_stream", c_void_p)]


class chfsi_stats(ctypes.Structure):
    _fields_ = [("loops", c_int32), ("filtered_vectors", c_int32), ("converged", c_int32),
                ("accept_rounds", c_int32), ("matvecs", c_int64), ("filter_matvecs", c_int64),
                ("launches", c_int64), ("filter_matvecs_fp64", c_int64),
                ("tensor_flops", c_double), ("max_resid", c_double),
                ("lanczos_upper", c_double), ("t_reduce_ms", c_double), ("t_lanczos_ms", c_double),
                ("t_filter_ms", c_double), ("t_qr_ms", c_double), ("t_rr_ms", c_double),
                ("t_resid_ms", c_double), ("t_total_ms", c_double), ("t_filter_gemm_ms", c_double),
                ("t_small_ms", c_double), ("t_eig_ms", c_double),
                ("filter_products", c_int64), ("filter_slice_bytes", c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_P = c_void_p
_SIGS = {
    "chfsi_default_opts": (None, [POINTER(chfsi_opts)]),
    "chfsi_create": (c_int32, [POINTER(c_void_p), c_int64, c_int32, POINTER(chfsi_opts)]),
    "chfsi_destroy": (None, [_P]),
    "chfsi_last_error": (c_char_p, [_P]),
    "chfsi_reset_warm_state": (c_int32, [_P]),
    "chfsi_get_state": (c_int32, [_P, POINTER(c_int64), POINTER(c_int32), _P, _P]),
    "chfsi_set_state": (c_int32, [_P, c_int64, c_int32, _P, c_int64, _P]),
    "chfsi_solve_next": (c_int32, [_P, c_int64, _P, c_int64, _P, c_int64, _P, c_int32, c_int32,
                                   c_int32, c_double, _P, _P, POINTER(chfsi_stats)]),
    "chfsi_solve_sequence": (c_int32, [_P, c_int32, c_int64, _P, _P, c_int64, _P, c_int32,
                                       c_int32, c_int32, c_double, _P, _P, POINTER(chfsi_stats)]),
    "chfsi_cholesky": (c_int32, [_P, c_int64, _P, c_int64, _P, c_int64]),
    "chfsi_reduce": (c_int32, [_P, c_int64, _P, c_int64, _P, c_int64, _P, c_int64]),
    "chfsi_lanczos": (c_int32, [_P, c_int64, _P, c_int64, c_int32, _P, POINTER(c_double),
                                POINTER(c_double), POINTER(c_double)]),
    "chfsi_filter": (c_int32, [_P, c_int64, c_int32, _P, c_int64, _P, c_int64, POINTER(c_int32),
                               c_double, c_double, c_double]),
    "chfsi_filter_split": (c_int32, [_P, c_int64, c_int32, _P, c_int64, _P, c_int64,
                                     POINTER(c_int32), c_double, c_double, c_double, c_int32]),
    "chfsi_orthonormalize": (c_int32, [_P, c_int64, c_int32, _P, c_int64, c_int32, _P, c_int64]),
    "chfsi_rayleigh_ritz": (c_int32, [_P, c_int64, c_int32, _P, c_int64, _P, c_int64, _P, c_int64,
                                      _P]),
    "chfsi_residuals": (c_int32, [_P, c_int64, c_int32, _P, c_int64, _P, c_int64, _P, _P]),
    "chfsi_degrees": (c_int32, [_P, c_int32, _P, _P, c_double, c_double, c_double, c_int32,
                                c_int32, c_int32, _P]),
    "chfsi_heev": (c_int32, [_P, c_int32, _P, c_int64, _P, _P, c_int64]),
    "chfsi_heev_df": (c_int32, [_P, c_int32, _P, c_int64, _P, _P, c_int64]),
    "chfsi_mlp_init": (None, [_P, c_uint64]),
    "chfsi_mlp_train": (c_int32, [_P, _P, _P, _P, c_int64, c_int32, c_int32, ctypes.c_float, c_uint64, _P]),
    "chfsi_mlp_gradient": (c_int32, [_P, _P, _P, _P, c_int64, _P, _P]),
    "chfsi_mlp_adam_epoch": (c_int32, [_P, _P, _P, _P, _P, _P, _P, _P, c_int64, c_int32, ctypes.c_float, _P]),
    "chfsi_mlp_predict": (c_int32, [_P, _P, _P, c_int64, _P]),
    "chfsi_set_degree_model": (c_int32, [_P, _P]),
    "chfsi_degree_log_start": (c_int32, [_P, c_int64]),
    "chfsi_degree_log_read": (c_int64, [_P, _P, c_int64]),
    "chfsi_batch_create": (c_int32, [POINTER(c_void_p), c_int32, c_int64, c_int32, POINTER(chfsi_opts)]),
    "chfsi_batch_destroy": (None, [_P]),
    "chfsi_batch_last_error": (c_char_p, [_P]),
    "chfsi_batch_solve": (c_int32, [_P, c_int32, c_int32, _P, _P, _P, c_int32, c_double, _P, _P, _P, _P, _P,
                                    _P]),
    "chfsi_deviation_angles": (c_int32, [_P, c_int64, c_int32, _P, c_int64, _P, c_int64, _P, c_int64,
                                         _P, _P]),
    "chfsi_heev_noalloc": (c_int32, [c_int32, _P, c_int64, _P, _P, c_int64, _P]),
    "chfsi_set_wait_limit": (c_int32, [_P, c_int64]),
    "chfsi_zgemm": (c_int32, [_P, c_char, c_char, c_int32, c_int32, c_int32, c_double, _P, c_int64,
                              _P, c_int64, c_double, _P, c_int64]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libchfsi.so (building it first if it is missing or stale)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.build() if build_if_missing else _build.LIB
    if not os.path.exists(path):
        raise RuntimeError(f"libchfsi.so not found at {path}; run paper_1206_3768_gb300.build")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


# ---------------------------------------------------------------------- helpers
def fortran(t: torch.Tensor) -> torch.Tensor:
    """Same matrix, column-major storage (no copy when it already is)."""
    if t.dim() == 1:
        return t.contiguous()
    if t.stride(0) == 1 and t.stride(1) >= max(1, t.shape[0]):
        return t
    return t.mT.contiguous().mT


def fortran_empty(rows: int, cols: int, device, dtype=torch.complex128) -> torch.Tensor:
    return torch.empty((cols, rows), dtype=dtype, device=device).mT


def _ld(t: torch.Tensor) -> int:
    if t.dim() == 2 and t.shape[1] > 1:
        return max(1, t.stride(1))
    return max(1, t.shape[0])  # one column (or a vector): its stride is irrelevant


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _check(ctx, rc: int):
    if rc != CHFSI_OK:
        msg = load().chfsi_last_error(ctx).decode() if ctx else ""
        raise ChfsiError(rc, msg)


def default_opts(**kw) -> chfsi_opts:
    o = chfsi_opts()
    load().chfsi_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


# ---------------------------------------------------------------------- context
_CUDA_STREAM_LEGACY = 0x1  # cudaStreamLegacy: the context's legacy default stream


def _stream_handle(stream) -> int:
    """Raw cudaStream_t for the library: torch's current stream unless one is given, so the
    library's work is ordered after torch's pending work on the same tensors (and torch's
    later work after the library's).  torch's default stream is the legacy NULL stream,
    passed as cudaStreamLegacy because a NULL handle asks the library for its own stream."""
    if stream is None:
        stream = torch.cuda.current_stream()
    h = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    return h if h else _CUDA_STREAM_LEGACY


def chfsi_create(n_max: int, blk_max: int, opts: chfsi_opts | None = None, stream=None, **kw):
    lib = load()
    o = opts if opts is not None else default_opts(**kw)
    if torch.cuda.is_available() or stream is not None:
        o.cuda_stream = ctypes.c_void_p(_stream_handle(stream))
    ctx = ctypes.c_void_p()
    rc = lib.chfsi_create(ctypes.byref(ctx), int(n_max), int(blk_max), ctypes.byref(o))
    if rc != CHFSI_OK:
        raise ChfsiError(rc, "chfsi_create failed")
    return ctx


def chfsi_destroy(ctx):
    load().chfsi_destroy(ctx)


def chfsi_last_error(ctx) -> str:
    return load().chfsi_last_error(ctx).decode()


def chfsi_reset_warm_state(ctx):
    _check(ctx, load().chfsi_reset_warm_state(ctx))


def chfsi_get_state(ctx, device="cuda"):
    """The warm state (x-coordinate Ritz vectors n x blk, Ritz values) or None."""
    n, blk = c_int64(0), c_int32(0)
    _check(ctx, load().chfsi_get_state(ctx, ctypes.byref(n), ctypes.byref(blk), None, None))
    if n.value == 0:
        return None
    X = fortran_empty(n.value, blk.value, torch.device(device))
    lam = torch.empty(blk.value, dtype=torch.float64)  # host
    _check(ctx, load().chfsi_get_state(ctx, ctypes.byref(n), ctypes.byref(blk), _ptr(X), _ptr(lam)))
    return X, lam


def chfsi_set_state(ctx, state):
    """Install a state from chfsi_get_state (None clears it)."""
    if state is None:
        _check(ctx, load().chfsi_set_state(ctx, 0, 0, None, 1, None))
        return
    X, lam = state
    Xf = fortran(X)
    lam = torch.as_tensor(lam, dtype=torch.float64).cpu().contiguous()
    _check(ctx, load().chfsi_set_state(ctx, Xf.shape[0], Xf.shape[1], _ptr(Xf), _ld(Xf), _ptr(lam)))


def chfsi_solve_next(ctx, A: torch.Tensor, B: torch.Tensor, nev: int, blk: int, deg: int,
                     tol: float = 1e-10, V0: torch.Tensor | None = None, out_device=None,
                     want_vectors: bool = True):
    """One problem.  Returns (evals [nev] float64, evecs [n, nev] complex128, stats dict)."""
    n = A.shape[0]
    dev = A.device if out_device is None else torch.device(out_device)
    Af, Bf = fortran(A), fortran(B)
    V0f = fortran(V0) if V0 is not None else None
    if V0f is not None and _ld(V0f) != n:
        V0f = V0f.mT.contiguous().mT  # ld must equal n
    evals = torch.empty(nev, dtype=torch.float64, device=dev)
    evecs = fortran_empty(n, nev, dev) if want_vectors else None
    st = chfsi_stats()
    rc = load().chfsi_solve_next(ctx, n, _ptr(Af), _ld(Af), _ptr(Bf), _ld(Bf), _ptr(V0f), nev, blk,
                                 deg, tol, _ptr(evals), _ptr(evecs), ctypes.byref(st))
    if rc not in (CHFSI_OK, CHFSI_ENOCONV):
        _check(ctx, rc)
    out = (evals, evecs, st.as_dict())
    if rc == CHFSI_ENOCONV:
        err = ChfsiError(rc, chfsi_last_error(ctx))
        err.partial = out
        raise err
    return out


def chfsi_solve_sequence(ctx, As, Bs, nev: int, blk: int, deg: int, tol: float = 1e-10,
                         V0: torch.Tensor | None = None, want_vectors: bool = True):
    """N problems in order with warm starts.  As, Bs: lists of n x n tensors (same device,
    column-major with a common leading dimension).  Returns (evals [N, nev], list of evecs,
    list of stats dicts)."""
    N = len(As)
    n = As[0].shape[0]
    Af = [fortran(a) for a in As]
    Bf = [fortran(b) for b in Bs]
    ld = _ld(Af[0])
    if any(_ld(x) != ld for x in Af + Bf):
        raise ValueError("all matrices must share one leading dimension")
    dev = As[0].device
    evals = torch.empty((N, nev), dtype=torch.float64, device="cpu")
    evecs = [fortran_empty(n, nev, dev) for _ in range(N)] if want_vectors else None
    Ap = (c_void_p * N)(*[a.data_ptr() for a in Af])
    Bp = (c_void_p * N)(*[b.data_ptr() for b in Bf])
    Ep = (c_void_p * N)(*[e.data_ptr() for e in evecs]) if evecs else None
    V0f = fortran(V0) if V0 is not None else None
    if V0f is not None and _ld(V0f) != n:
        V0f = V0f.mT.contiguous().mT
    sts = (chfsi_stats * N)()
    rc = load().chfsi_solve_sequence(ctx, N, n, Ap, Bp, ld, _ptr(V0f), nev, blk, deg, tol,
                                     _ptr(evals), Ep, sts)
    _check(ctx, rc)
    return evals, evecs, [s.as_dict() for s in sts]


# ---------------------------------------------------------------------- steps
def chfsi_cholesky(ctx, B: torch.Tensor) -> torch.Tensor:
    n = B.shape[0]
    Bf = fortran(B)
    L = fortran_empty(n, n, B.device)
    _check(ctx, load().chfsi_cholesky(ctx, n, _ptr(Bf), _ld(Bf), _ptr(L), _ld(L)))
    return L


def chfsi_reduce(ctx, A: torch.Tensor, L: torch.Tensor) -> torch.Tensor:
    n = A.shape[0]
    Af, Lf = fortran(A), fortran(L)
    H = fortran_empty(n, n, A.device)
    _check(ctx, load().chfsi_reduce(ctx, n, _ptr(Af), _ld(Af), _ptr(Lf), _ld(Lf), _ptr(H), _ld(H)))
    return H


def chfsi_lanczos(ctx, H: torch.Tensor, k: int, v0: torch.Tensor | None = None):
    n = H.shape[0]
    Hf = fortran(H)
    up, tmin, tmax = c_double(), c_double(), c_double()
    v = v0.contiguous() if v0 is not None else None
    _check(ctx, load().chfsi_lanczos(ctx, n, _ptr(Hf), _ld(Hf), k, _ptr(v), ctypes.byref(up),
                                     ctypes.byref(tmin), ctypes.byref(tmax)))
    return up.value, tmin.value, tmax.value


def chfsi_filter(ctx, H: torch.Tensor, Y: torch.Tensor, degrees, a0: float, a: float, b: float):
    n, m = Y.shape
    Hf = fortran(H)
    Yf = fortran(Y).clone()
    degs = (c_int32 * m)(*[int(d) for d in degrees])
    _check(ctx, load().chfsi_filter(ctx, n, m, _ptr(Hf), _ld(Hf), _ptr(Yf), _ld(Yf), degs, a0, a, b))
    return Yf


def chfsi_filter_split(ctx, H: torch.Tensor, Y: torch.Tensor, degrees, a0: float, a: float,
                       b: float, slices: int = 7):
    n, m = Y.shape
    Hf = fortran(H)
    Yf = fortran(Y).clone()
    degs = (c_int32 * m)(*[int(d) for d in degrees])
    _check(ctx, load().chfsi_filter_split(ctx, n, m, _ptr(Hf), _ld(Hf), _ptr(Yf), _ld(Yf), degs, a0,
                                          a, b, slices))
    return Yf


def chfsi_orthonormalize(ctx, Y: torch.Tensor, YL: torch.Tensor | None = None):
    n, m = Y.shape
    Yf = fortran(Y.clone())
    k = 0 if YL is None else YL.shape[1]
    YLf = fortran(YL) if YL is not None else None
    _check(ctx, load().chfsi_orthonormalize(ctx, n, m, _ptr(Yf), _ld(Yf), k, _ptr(YLf),
                                            _ld(YLf) if YLf is not None else n))
    return Yf


def chfsi_rayleigh_ritz(ctx, H: torch.Tensor, Y: torch.Tensor):
    n, m = Y.shape
    Hf = fortran(H)
    Yf = fortran(Y.clone())
    HY = fortran_empty(n, m, Y.device)
    theta = torch.empty(m, dtype=torch.float64, device=Y.device)
    _check(ctx, load().chfsi_rayleigh_ritz(ctx, n, m, _ptr(Hf), _ld(Hf), _ptr(Yf), _ld(Yf),
                                           _ptr(HY), _ld(HY), _ptr(theta)))
    return theta, Yf, HY


def chfsi_residuals(ctx, HY: torch.Tensor, Y: torch.Tensor, theta: torch.Tensor):
    n, m = Y.shape
    HYf, Yf = fortran(HY), fortran(Y)
    r = torch.empty(m, dtype=torch.float64, device=Y.device)
    _check(ctx, load().chfsi_residuals(ctx, n, m, _ptr(HYf), _ld(HYf), _ptr(Yf), _ld(Yf),
                                       _ptr(theta.contiguous()), _ptr(r)))
    return r


def chfsi_degrees(ctx, theta: torch.Tensor, r: torch.Tensor, a: float, b: float, tau: float,
                  dmin: int, dmax: int, n_wanted: int):
    m = theta.shape[0]
    d = torch.empty(m, dtype=torch.int32, device=theta.device)
    _check(ctx, load().chfsi_degrees(ctx, m, _ptr(theta.contiguous()), _ptr(r.contiguous()), a, b,
                                     tau, dmin, dmax, n_wanted, _ptr(d)))
    return d


def chfsi_deviation_angles(ctx, X_prev: torch.Tensor, X_cur: torch.Tensor, B: torch.Tensor):
    """Deviation angles theta_i between x_prev_i and its associated current vector
    x_cur[:, assoc[i]] in the B-inner product (Section 2.2, Fig. 1).  Returns (theta, assoc)."""
    n, k = X_prev.shape
    Pf, Cf, Bf = fortran(X_prev), fortran(X_cur), fortran(B)
    theta = torch.empty(k, dtype=torch.float64, device=X_prev.device)
    assoc = torch.empty(k, dtype=torch.int32, device=X_prev.device)
    _check(ctx, load().chfsi_deviation_angles(ctx, n, k, _ptr(Pf), _ld(Pf), _ptr(Cf), _ld(Cf), _ptr(Bf),
                                              _ld(Bf), _ptr(theta), _ptr(assoc)))
    return theta, assoc


def chfsi_heev(ctx, G: torch.Tensor):
    m = G.shape[0]
    Gf = fortran(G)
    w = torch.empty(m, dtype=torch.float64, device=G.device)
    V = fortran_empty(m, m, G.device)
    _check(ctx, load().chfsi_heev(ctx, m, _ptr(Gf), _ld(Gf), _ptr(w), _ptr(V), _ld(V)))
    return w, V


def chfsi_heev_df(ctx, G: torch.Tensor):
    m = G.shape[0]
    Gf = fortran(G)
    w = torch.empty(m, dtype=torch.float64, device=G.device)
    V = fortran_empty(m, m, G.device)
    _check(ctx, load().chfsi_heev_df(ctx, m, _ptr(Gf), _ld(Gf), _ptr(w), _ptr(V), _ld(V)))
    return w, V


def chfsi_set_wait_limit(ctx, polls: int):
    _check(ctx, load().chfsi_set_wait_limit(ctx, int(polls)))


HEEV_NOALLOC_MAX = 128


def chfsi_heev_noalloc(G: torch.Tensor, stream=None):
    """Eigen-decomposition without a context or any device allocation by the library
    (scratch in a fixed device array; m <= 128).  The output tensors are allocated here by
    torch, as a caller of the C entry point would provide them.  The library works on the
    current device, so the call is made with G's device current and, by default, on that
    device's current torch stream."""
    if not (isinstance(G, torch.Tensor) and G.is_cuda and G.dtype == torch.complex128
            and G.dim() == 2 and G.shape[0] == G.shape[1]):
        raise ValueError("G must be a square complex128 CUDA tensor")
    m = G.shape[0]
    with torch.cuda.device(G.device):
        Gf = fortran(G)
        w = torch.empty(m, dtype=torch.float64, device=G.device)
        V = fortran_empty(m, m, G.device)
        s = ctypes.c_void_p(_stream_handle(stream if stream is not None
                                           else torch.cuda.current_stream(G.device)))
        rc = load().chfsi_heev_noalloc(m, _ptr(Gf), _ld(Gf), _ptr(w), _ptr(V), _ld(V), s)
    if rc != CHFSI_OK:
        raise ChfsiError(rc, f"chfsi_heev_noalloc(m={m}) failed")
    return w, V


def chfsi_zgemm(ctx, opa: str, opb: str, alpha: float, A: torch.Tensor, B: torch.Tensor,
                beta: float = 0.0, C: torch.Tensor | None = None):
    Af, Bf = fortran(A), fortran(B)
    M = A.shape[0] if opa == "N" else A.shape[1]
    K = A.shape[1] if opa == "N" else A.shape[0]
    N = B.shape[1] if opb == "N" else B.shape[0]
    if C is None:
        C = fortran_empty(M, N, A.device)
        C.zero_()
    else:
        C = fortran(C.clone())
    _check(ctx, load().chfsi_zgemm(ctx, opa.encode(), opb.encode(), M, N, K, alpha, _ptr(Af),
                                   _ld(Af), _ptr(Bf), _ld(Bf), beta, _ptr(C), _ld(C)))
    return C


def _f32(x):
    import numpy as np

    return np.ascontiguousarray(np.asarray(x, dtype=np.float32))


def chfsi_mlp_init(seed: int = 12063768) -> chfsi_mlp:
    m = chfsi_mlp()
    load().chfsi_mlp_init(ctypes.byref(m), seed)
    return m


def chfsi_mlp_train(ctx, model: chfsi_mlp, X, z, epochs: int, batch: int = 256, lr: float = 1e-3,
                    seed: int = 1) -> float:
    """Train in place on host data X (n x MLP_IN) and targets z (n); returns the last epoch's
    loss."""
    X, z = _f32(X), _f32(z)
    loss = ctypes.c_float()
    _check(ctx, load().chfsi_mlp_train(ctx, ctypes.byref(model), X.ctypes.data, z.ctypes.data, len(z),
                                       epochs, batch, lr, seed, ctypes.byref(loss)))
    return float(loss.value)


def chfsi_mlp_gradient(ctx, model: chfsi_mlp, X, z):
    """(gradient of the mean squared error over all samples [MLP_NPARAM], loss)."""
    import numpy as np

    X, z = _f32(X), _f32(z)
    g = np.empty(MLP_NPARAM, dtype=np.float32)
    loss = ctypes.c_float()
    _check(ctx, load().chfsi_mlp_gradient(ctx, ctypes.byref(model), X.ctypes.data, z.ctypes.data, len(z),
                                          g.ctypes.data, ctypes.byref(loss)))
    return g, float(loss.value)


def chfsi_mlp_adam_epoch(ctx, model: chfsi_mlp, m1, m2, step: int, X, z, order, batch: int, lr: float):
    """One Adam epoch in the given sample order; model updated in place.  Returns
    (m1, m2, step, loss) with the updated moments (float32 arrays) and step counter."""
    import numpy as np

    X, z = _f32(X), _f32(z)
    m1, m2 = _f32(m1).copy(), _f32(m2).copy()
    order = np.ascontiguousarray(np.asarray(order, dtype=np.int32))
    st = ctypes.c_int32(int(step))
    loss = ctypes.c_float()
    _check(ctx, load().chfsi_mlp_adam_epoch(ctx, ctypes.byref(model), m1.ctypes.data, m2.ctypes.data,
                                            ctypes.byref(st), X.ctypes.data, z.ctypes.data, order.ctypes.data,
                                            len(z), int(batch), float(lr), ctypes.byref(loss)))
    return m1, m2, int(st.value), float(loss.value)


def chfsi_mlp_predict(ctx, model: chfsi_mlp, X):
    import numpy as np

    X = _f32(X)
    y = np.empty(X.shape[0], dtype=np.float32)
    _check(ctx, load().chfsi_mlp_predict(ctx, ctypes.byref(model), X.ctypes.data, X.shape[0], y.ctypes.data))
    return y


def chfsi_set_degree_model(ctx, model: chfsi_mlp | None):
    _check(ctx, load().chfsi_set_degree_model(ctx, ctypes.byref(model) if model is not None else None))


def chfsi_degree_log_start(ctx, capacity: int):
    _check(ctx, load().chfsi_degree_log_start(ctx, capacity))


def chfsi_degree_log_read(ctx):
    """All logged records as an array [count, DEGREE_LOG_FIELDS]: problem, loop, g, i, m, theta,
    r, tau, d, c, e, r_next, x0 .. x7."""
    import numpy as np

    lib = load()
    cnt = lib.chfsi_degree_log_read(ctx, None, 0)
    out = np.empty((max(cnt, 0), DEGREE_LOG_FIELDS), dtype=np.float64)
    if cnt > 0:
        lib.chfsi_degree_log_read(ctx, out.ctypes.data, cnt)
    return out


def chfsi_batch_create(workers: int, n_max: int, blk_max: int, **kw):
    o = default_opts(**kw)
    ptr = ctypes.c_void_p()
    rc = load().chfsi_batch_create(ctypes.byref(ptr), int(workers), int(n_max), int(blk_max),
                                   ctypes.byref(o))
    if rc != CHFSI_OK:
        raise ChfsiError(rc, "chfsi_batch_create failed")
    return ptr


def chfsi_batch_destroy(batch):
    load().chfsi_batch_destroy(batch)


def chfsi_batch_last_error(batch) -> str:
    return load().chfsi_batch_last_error(batch).decode()


def chfsi_batch_solve(batch, seqs, nev, blk, deg: int, tol: float = 1e-10, want_vectors: bool = True):
    """K independent sequences on a batch.  seqs: list of (As, Bs) per sequence (N problems
    each, lists of n_s x n_s tensors, one device and leading dimension per sequence); nev,
    blk: lists.  Returns a list of (evals [N, nev_s], evecs list or None, stats dicts)."""
    return Batch.solve_on(batch, seqs, nev, blk, deg, tol, want_vectors)


class Batch:
    """Several contexts (own streams, one host worker thread each) solving independent
    sequences of uneven sizes concurrently (chfsi_batch_*)."""

    def __init__(self, workers: int, n_max: int, blk_max: int, **kw):
        self.ptr = chfsi_batch_create(workers, n_max, blk_max, **kw)

    def solve(self, seqs, nev, blk, deg: int, tol: float = 1e-10, want_vectors: bool = True):
        return Batch.solve_on(self.ptr, seqs, nev, blk, deg, tol, want_vectors)

    @staticmethod
    def solve_on(ptr, seqs, nev, blk, deg: int, tol: float = 1e-10, want_vectors: bool = True):
        K = len(seqs)
        N = len(seqs[0][0])
        if any(len(a) != N or len(b) != N for a, b in seqs):
            raise ValueError("every sequence needs the same number of problems")
        keep = []
        n_arr = (c_int64 * K)()
        ld_arr = (c_int64 * K)()
        Ap = (c_void_p * (K * N))()
        Bp = (c_void_p * (K * N))()
        Ev = (c_void_p * K)()
        Xp = (c_void_p * (K * N))() if want_vectors else None
        out = []
        for s_i, (As, Bs) in enumerate(seqs):
            Af = [fortran(a) for a in As]
            Bf = [fortran(b) for b in Bs]
            ld = _ld(Af[0])
            if any(_ld(x) != ld for x in Af + Bf):
                raise ValueError("matrices of one sequence must share one leading dimension")
            n = Af[0].shape[0]
            n_arr[s_i], ld_arr[s_i] = n, ld
            ev = torch.empty((N, nev[s_i]), dtype=torch.float64, device="cpu")
            Ev[s_i] = ev.data_ptr()
            X = [fortran_empty(n, nev[s_i], Af[0].device) for _ in range(N)] if want_vectors else None
            for l in range(N):
                Ap[s_i * N + l] = Af[l].data_ptr()
                Bp[s_i * N + l] = Bf[l].data_ptr()
                if X is not None:
                    Xp[s_i * N + l] = X[l].data_ptr()
            keep += [Af, Bf]
            out.append((ev, X))
        nev_arr = (c_int32 * K)(*nev)
        blk_arr = (c_int32 * K)(*blk)
        sts = (chfsi_stats * (K * N))()
        if torch.cuda.is_available():
            torch.cuda.synchronize()  # inputs written on torch's streams; the batch has its own
        lib = load()
        rc = lib.chfsi_batch_solve(ptr, K, N, n_arr, nev_arr, blk_arr, deg, tol, Ap, Bp, ld_arr, Ev, Xp,
                                   sts)
        if rc != CHFSI_OK:
            raise ChfsiError(rc, lib.chfsi_batch_last_error(ptr).decode())
        return [(ev, X, [sts[s_i * N + l].as_dict() for l in range(N)])
                for s_i, (ev, X) in enumerate(out)]

    def close(self):
        if self.ptr:
            chfsi_batch_destroy(self.ptr)
            self.ptr = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver:
    """Context manager owning one chfsi context."""

    def __init__(self, n_max: int, blk_max: int, stream=None, **opts):
        self.ctx = chfsi_create(n_max, blk_max, stream=stream, **opts)

    def close(self):
        if self.ctx:
            chfsi_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
