"""Thin Python binding of libpluqmodp (argument marshalling only).

Every step of the factorization runs in the CUDA library; this module only
checks tensor dtypes/devices, passes raw device pointers and the current torch
stream through ctypes, and wraps the outputs.  Residues travel as torch.int32
tensors (p < 2^31, so every residue is a non-negative int32 with the bits of
the library's uint32).  If the library is missing or a GPU is absent the calls
raise; there is no fallback.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libpluqmodp.so")

FORM_AUTO, FORM_FP64, FORM_LIMB_F16 = 0, 1, 2
FORMS = {"auto": FORM_AUTO, "fp64": FORM_FP64, "limb": FORM_LIMB_F16, "limb_f16": FORM_LIMB_F16}

STATUS = {
    0: "ok", -1: "invalid argument", -2: "p is not prime", -3: "p out of range",
    -4: "matrix entry >= p", -5: "fgemm form unsupported for this p",
    -6: "device workspace allocation failed", -7: "CUDA error", -8: "device wait timed out",
    -9: "exceeds the fixed scratch of the non-allocating entry point",
}

_lib = None

# Exported C symbols (kept in sync with include/pluqmodp.h).
SYMBOLS = [
    "pluq_create", "pluq_destroy", "pluq_modp", "echelon_modp", "rank_profile_modp",
    "fgemm_modp", "pluq_modp_batched", "pluq_last_rank", "pluq_set_tuning", "pluq_last_stats",
    "pluq_status_string", "pluq_profile_enable", "pluq_profile_read", "pluq_set_leaf",
    "fgemm_modp_noalloc", "pluq_set_option", "pluq_autotune", "column_echelon_modp",
    "rank_profile_modp_batched", "echelon_modp_batched", "pluq_sync_status",
]


class PluqError(RuntimeError):
    def __init__(self, status: int, where: str):
        super().__init__(f"{where}: {STATUS.get(status, status)} ({status})")
        self.status = status


def load():
    """Load libpluqmodp.so (built in-tree by build.py); raise if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                           "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(LIB_PATH)
    vp, i64, u32, i32 = ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint32, ctypes.c_int
    sig = {
        "pluq_create": [ctypes.POINTER(vp), i32],
        "pluq_destroy": [vp],
        "pluq_modp": [vp, u32, i64, i64, vp, i64, vp, vp, vp, vp, vp, i32, vp],
        "echelon_modp": [vp, u32, i64, i64, vp, i64, vp, i64, vp, vp, i32, vp],
        "column_echelon_modp": [vp, u32, i64, i64, vp, i64, vp, i64, vp, vp, i32, vp],
        "rank_profile_modp": [vp, u32, i64, i64, vp, i64, vp, vp, vp, vp, i32, vp],
        "fgemm_modp": [vp, u32, i64, i64, i64, vp, i64, vp, i64, vp, i64, i32, vp],
        "pluq_modp_batched": [vp, u32, ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, i32, vp],
        "rank_profile_modp_batched": [vp, u32, ctypes.c_int32, vp, vp, vp, vp, vp, vp, vp, vp, i32,
                                      vp],
        "pluq_last_rank": [vp, vp],
        "pluq_sync_status": [vp],
        "pluq_set_tuning": [vp, i32, i32, i32],
        "pluq_last_stats": [vp, vp, vp, vp],
        "pluq_status_string": [i32],
        "pluq_profile_enable": [vp, i32],
        "pluq_set_leaf": [vp, i32],
        "pluq_set_option": [vp, i32, i32],
        "fgemm_modp_noalloc": [u32, i64, i64, i64, vp, i64, vp, i64, vp, i64, vp],
        "pluq_profile_read": [vp, i32, vp, vp, vp, vp, vp],
        "pluq_autotune": [vp, u32, i64, i64, vp, i64, i32, vp, ctypes.c_double, vp, vp],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "pluq_status_string" else ctypes.c_int
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise PluqError(status, where)


def _dev_ptr(t: torch.Tensor | None, dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must have dtype {dtype}, got {t.dtype}")
    return ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream) -> ctypes.c_void_p:
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _form(form) -> int:
    return FORMS[form] if isinstance(form, str) else int(form)


def _matrix_args(A: torch.Tensor, name="A"):
    if A.dim() != 2 or A.dtype != torch.int32:
        raise ValueError(f"{name} must be a 2-D torch.int32 tensor of residues")
    if A.stride(1) != 1 and A.numel() > 0:
        raise ValueError(f"{name} must be row-major (unit column stride)")
    m, n = A.shape
    ld = A.stride(0) if m > 1 else max(n, 1)
    return m, n, max(ld, n, 1)


class Context:
    """Owns a library context (device workspace) bound to one CUDA device."""

    def __init__(self, device: int | None = None):
        lib = load()
        if device is None:
            device = torch.cuda.current_device()
        self.device = device
        h = ctypes.c_void_p()
        _check(lib.pluq_create(ctypes.byref(h), device), "pluq_create")
        self.handle = h

    def close(self):
        if getattr(self, "handle", None):
            load().pluq_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    OPTIONS = {"leaf_dim": 1, "leaf_kind": 2, "tile_m": 3, "tile_n": 4, "trsm_block": 5,
               "chain_rows": 6, "fork_depth": 7, "use_tuned": 8, "thin_gemm": 9,
               "decomposition": 10, "slab_rows": 11, "wait_limit_us": 12, "workspace_mb": 13,
               "winograd_min": 14, "fgemm_tile": 15, "trsm_strip": 16,
               "fused_kmax": 17, "diag_inverses": 18,
               "batch_slab": 19, "lookahead": 20}

    def set_option(self, name: str, value: int):
        """Set a recursion option (see PLUQ_OPT_* in include/pluqmodp.h)."""
        _check(load().pluq_set_option(self.handle, self.OPTIONS[name], int(value)),
               "pluq_set_option")

    def set_leaf(self, leaf_dim: int):
        """Largest block factored by one cooperative leaf launch (0: one-CTA tiles only)."""
        _check(load().pluq_set_leaf(self.handle, leaf_dim), "pluq_set_leaf")

    def set_tuning(self, bm: int = 0, bn: int = 0, trsm_block: int = 0):
        _check(load().pluq_set_tuning(self.handle, bm, bn, trsm_block), "pluq_set_tuning")

    PROFILE_CLASSES = ["base", "fgemm", "pack", "trsm", "perm", "index", "other", "thin"]

    def profile(self, enable: bool = True):
        """Reset the per-class launch counters; with enable, time every launch."""
        _check(load().pluq_profile_enable(self.handle, 1 if enable else 0), "pluq_profile_enable")

    def profile_read(self) -> dict:
        """Per kernel class: launches, device ms, algorithmic flops/bytes, tensor flops."""
        out = {}
        for k, name in enumerate(self.PROFILE_CLASSES):
            nl, ms, fl, by, tf = (ctypes.c_int64(), ctypes.c_double(), ctypes.c_double(),
                                  ctypes.c_double(), ctypes.c_double())
            _check(load().pluq_profile_read(self.handle, k, ctypes.byref(nl), ctypes.byref(ms),
                                            ctypes.byref(fl), ctypes.byref(by), ctypes.byref(tf)),
                   "pluq_profile_read")
            out[name] = {"launches": nl.value, "ms": ms.value, "flops": fl.value,
                         "bytes": by.value, "tensor_flops": tf.value}
        return out

    LEAF_KINDS = {0: "barrier", 1: "wavefront", 2: "per-leaf", 3: "cluster", 4: "tile"}

    def autotune(self, A: torch.Tensor, p: int, form="limb", budget_ms: float = 0.0,
                 stream=None) -> dict:
        """Time candidate recursion schedules on copies of A and keep the fastest for
        A's (p, shape, form) in this context (pluq_autotune); A is not modified."""
        m, n, ld = _matrix_args(A)
        chosen = (ctypes.c_int32 * 4)()
        best = ctypes.c_double()
        _check(load().pluq_autotune(self.handle, p, m, n, ctypes.c_void_p(A.data_ptr()), ld,
                                    _form(form), _stream_handle(stream), float(budget_ms), chosen,
                                    ctypes.byref(best)), "pluq_autotune")
        return {"leaf_dim": chosen[0], "leaf_kind": self.LEAF_KINDS.get(chosen[1], chosen[1]),
                "fork_depth": chosen[2], "fgemm_tile": chosen[3], "ms": best.value}

    def last_stats(self) -> dict:
        a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        _check(load().pluq_last_stats(self.handle, ctypes.byref(a), ctypes.byref(b),
                                      ctypes.byref(c)), "pluq_last_stats")
        return {"base_cases": a.value, "nodes": b.value, "fgemm_calls": c.value}


_default_ctx: dict[int, Context] = {}


def default_context(device: int | None = None) -> Context:
    d = torch.cuda.current_device() if device is None else device
    if d not in _default_ctx:
        _default_ctx[d] = Context(d)
    return _default_ctx[d]


@dataclass
class PLUQResult:
    rank: int
    P: torch.Tensor
    Q: torch.Tensor
    LU: torch.Tensor
    rrp: torch.Tensor
    crp: torch.Tensor


def pluq_modp(A: torch.Tensor, p: int, form="auto", ctx: Context | None = None, stream=None,
              profiles: bool = True) -> PLUQResult:
    """In-place PLUQ of A (CUDA int32 residues); A becomes the compressed L\\U."""
    ctx = ctx or default_context(A.device.index)
    m, n, lda = _matrix_args(A)
    dev = A.device
    P = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    Q = torch.empty(max(n, 1), dtype=torch.int32, device=dev)
    rk = torch.zeros(1, dtype=torch.int64, device=dev)
    rmax = max(min(m, n), 1)
    rrp = torch.empty(rmax, dtype=torch.int32, device=dev) if profiles else None
    crp = torch.empty(rmax, dtype=torch.int32, device=dev) if profiles else None
    st = load().pluq_modp(ctx.handle, p, m, n, _dev_ptr(A), lda, _dev_ptr(P), _dev_ptr(Q),
                          _dev_ptr(rk), _dev_ptr(rrp), _dev_ptr(crp), _form(form),
                          _stream_handle(stream))
    _check(st, "pluq_modp")
    r = last_rank(ctx)
    return PLUQResult(r, P[:m], Q[:n], A, rrp[:r] if profiles else None,
                      crp[:r] if profiles else None)


def echelon_modp(A: torch.Tensor, p: int, form="auto", ctx: Context | None = None, stream=None):
    """Reduced row echelon form of A: returns (rank, R (r x n int32), crp)."""
    ctx = ctx or default_context(A.device.index)
    m, n, lda = _matrix_args(A)
    dev = A.device
    rmax = max(min(m, n), 1)
    R = torch.zeros((rmax, max(n, 1)), dtype=torch.int32, device=dev)
    crp = torch.empty(rmax, dtype=torch.int32, device=dev)
    st = load().echelon_modp(ctx.handle, p, m, n, _dev_ptr(A), lda, _dev_ptr(R), max(n, 1), None,
                             _dev_ptr(crp), _form(form), _stream_handle(stream))
    _check(st, "echelon_modp")
    r = last_rank(ctx)
    return r, R[:r, :n], crp[:r]


def column_echelon_modp(A: torch.Tensor, p: int, form="auto", ctx: Context | None = None,
                        stream=None):
    """Reduced column echelon form RREF(A^T)^T: returns (rank, E (m x r int32), rrp)."""
    ctx = ctx or default_context(A.device.index)
    m, n, lda = _matrix_args(A)
    dev = A.device
    rmax = max(min(m, n), 1)
    E = torch.zeros((max(m, 1), rmax), dtype=torch.int32, device=dev)
    rrp = torch.empty(rmax, dtype=torch.int32, device=dev)
    st = load().column_echelon_modp(ctx.handle, p, m, n, _dev_ptr(A), lda, _dev_ptr(E), rmax,
                                    None, _dev_ptr(rrp), _form(form), _stream_handle(stream))
    _check(st, "column_echelon_modp")
    r = last_rank(ctx)
    return r, E[:m, :r], rrp[:r]


def rank_profile_modp(A: torch.Tensor, p: int, form="auto", ctx: Context | None = None,
                      stream=None):
    """Rank, row and column rank profiles, rank profile matrix (row -> column or -1)."""
    ctx = ctx or default_context(A.device.index)
    m, n, lda = _matrix_args(A)
    dev = A.device
    rmax = max(min(m, n), 1)
    rrp = torch.empty(rmax, dtype=torch.int32, device=dev)
    crp = torch.empty(rmax, dtype=torch.int32, device=dev)
    rpm = torch.empty(max(m, 1), dtype=torch.int32, device=dev)
    st = load().rank_profile_modp(ctx.handle, p, m, n, _dev_ptr(A), lda, None, _dev_ptr(rrp),
                                  _dev_ptr(crp), _dev_ptr(rpm), _form(form),
                                  _stream_handle(stream))
    _check(st, "rank_profile_modp")
    r = last_rank(ctx)
    return r, rrp[:r], crp[:r], rpm[:m]


def fgemm_modp(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, p: int, form="auto",
               ctx: Context | None = None, stream=None) -> torch.Tensor:
    """C <- C - A B mod p, in place (CUDA int32 residues)."""
    ctx = ctx or default_context(C.device.index)
    M, K, lda = _matrix_args(A, "A")
    K2, N, ldb = _matrix_args(B, "B")
    M2, N2, ldc = _matrix_args(C, "C")
    if K2 != K or M2 != M or N2 != N:
        raise ValueError("shape mismatch")
    st = load().fgemm_modp(ctx.handle, p, M, N, K, _dev_ptr(A), lda, _dev_ptr(B), ldb,
                           _dev_ptr(C), ldc, _form(form), _stream_handle(stream))
    _check(st, "fgemm_modp")
    return C


def fgemm_modp_noalloc(C: torch.Tensor, A: torch.Tensor, B: torch.Tensor, p: int,
                       stream=None) -> torch.Tensor:
    """C <- C - A B mod p through the entry point that allocates no device memory.

    For callers that cannot allocate (the library uses a fixed 32 MiB device
    array instead of context workspace); concurrent calls on different
    streams race on that array.
    """
    M, K, lda = _matrix_args(A, "A")
    K2, N, ldb = _matrix_args(B, "B")
    M2, N2, ldc = _matrix_args(C, "C")
    if K2 != K or M2 != M or N2 != N:
        raise ValueError("shape mismatch")
    st = load().fgemm_modp_noalloc(p, M, N, K, _dev_ptr(A), lda, _dev_ptr(B), ldb, _dev_ptr(C),
                                   ldc, _stream_handle(stream))
    _check(st, "fgemm_modp_noalloc")
    return C


class BatchPlan:
    """Marshalled arguments of pluq_modp_batched for a fixed list of matrices.

    Builds the pointer/size arrays once (and the P, Q outputs) so that repeated
    calls on the same device buffers cost one C call each.
    """

    def __init__(self, As: list, p: int, form="auto", ctx: Context | None = None):
        self.ctx = ctx or default_context(As[0].device.index)
        self.p, self.form, self.As = p, _form(form), As
        b = self.batch = len(As)
        self.ms = (ctypes.c_int64 * b)()
        self.ns = (ctypes.c_int64 * b)()
        self.lds = (ctypes.c_int64 * b)()
        self.aptr = (ctypes.c_void_p * b)()
        self.pptr = (ctypes.c_void_p * b)()
        self.qptr = (ctypes.c_void_p * b)()
        self.ranks = (ctypes.c_int64 * b)()
        self.status = (ctypes.c_int32 * b)()
        self.Ps, self.Qs = [], []
        for i, A in enumerate(As):
            m, n, ld = _matrix_args(A)
            self.ms[i], self.ns[i], self.lds[i] = m, n, ld
            self.aptr[i] = A.data_ptr() if A.numel() else None
            P = torch.empty(max(m, 1), dtype=torch.int32, device=A.device)
            Q = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
            self.Ps.append(P)
            self.Qs.append(Q)
            self.pptr[i] = P.data_ptr()
            self.qptr[i] = Q.data_ptr()

    def run(self, stream=None) -> int:
        """One batched factorization; returns the C status (per-matrix in .status)."""
        return load().pluq_modp_batched(self.ctx.handle, self.p, self.batch, self.ms, self.ns,
                                        self.aptr, self.lds, self.pptr, self.qptr, self.ranks,
                                        self.status, self.form, _stream_handle(stream))


def pluq_modp_batched(As: list, p: int, form="auto", ctx: Context | None = None, stream=None,
                      return_status: bool = False):
    """Batched in-place PLUQ of a list of CUDA int32 matrices: (ranks, Ps, Qs[, status]).

    With return_status, per-matrix status codes are returned instead of
    raising on the first failure.
    """
    if not As:
        return ([], [], [], []) if return_status else ([], [], [])
    ctx = ctx or default_context(As[0].device.index)
    b = len(As)
    ms = (ctypes.c_int64 * b)()
    ns = (ctypes.c_int64 * b)()
    lds = (ctypes.c_int64 * b)()
    aptr = (ctypes.c_void_p * b)()
    pptr = (ctypes.c_void_p * b)()
    qptr = (ctypes.c_void_p * b)()
    ranks = (ctypes.c_int64 * b)()
    status = (ctypes.c_int32 * b)()
    Ps, Qs = [], []
    for i, A in enumerate(As):
        m, n, ld = _matrix_args(A)
        ms[i], ns[i], lds[i] = m, n, ld
        aptr[i] = A.data_ptr() if A.numel() else None
        P = torch.empty(max(m, 1), dtype=torch.int32, device=A.device)
        Q = torch.empty(max(n, 1), dtype=torch.int32, device=A.device)
        Ps.append(P)
        Qs.append(Q)
        pptr[i] = P.data_ptr()
        qptr[i] = Q.data_ptr()
    st = load().pluq_modp_batched(ctx.handle, p, b, ms, ns, aptr, lds, pptr, qptr, ranks, status,
                                  _form(form), _stream_handle(stream))
    outs = (list(ranks), [P[:ms[i]] for i, P in enumerate(Ps)],
            [Q[:ns[i]] for i, Q in enumerate(Qs)])
    if return_status:
        return outs + (list(status),)
    _check(st, "pluq_modp_batched")
    return outs


def echelon_modp_batched(As: list, p: int, form="auto", ctx: Context | None = None,
                         stream=None, return_status: bool = False):
    """Reduced row echelon forms of a list of CUDA int32 matrices (not modified):
    (ranks, Rs (r x n each), crps[, status])."""
    if not As:
        return ([], [], [], []) if return_status else ([], [], [])
    ctx = ctx or default_context(As[0].device.index)
    b = len(As)
    ms = (ctypes.c_int64 * b)()
    ns = (ctypes.c_int64 * b)()
    lds = (ctypes.c_int64 * b)()
    ldr = (ctypes.c_int64 * b)()
    aptr = (ctypes.c_void_p * b)()
    rptr = (ctypes.c_void_p * b)()
    cptr = (ctypes.c_void_p * b)()
    ranks = (ctypes.c_int64 * b)()
    status = (ctypes.c_int32 * b)()
    Rs, Cs = [], []
    for i, A in enumerate(As):
        m, n, ld = _matrix_args(A)
        ms[i], ns[i], lds[i], ldr[i] = m, n, ld, max(n, 1)
        aptr[i] = A.data_ptr() if A.numel() else None
        R = torch.zeros((max(min(m, n), 1), max(n, 1)), dtype=torch.int32, device=A.device)
        cc = torch.empty(max(min(m, n), 1), dtype=torch.int32, device=A.device)
        Rs.append(R)
        Cs.append(cc)
        rptr[i] = R.data_ptr()
        cptr[i] = cc.data_ptr()
    st = load().echelon_modp_batched(ctx.handle, p, b, ms, ns, aptr, lds, rptr, ldr, cptr, ranks,
                                     status, _form(form), _stream_handle(stream))
    rk = list(ranks)
    outs = (rk, [Rs[i][:max(rk[i], 0), :ns[i]] for i in range(b)],
            [Cs[i][:max(rk[i], 0)] for i in range(b)])
    if return_status:
        return outs + (list(status),)
    _check(st, "echelon_modp_batched")
    return outs


def rank_profile_modp_batched(As: list, p: int, form="auto", ctx: Context | None = None,
                              stream=None, return_status: bool = False):
    """Ranks and sorted row / column rank profiles of a list of CUDA int32 matrices
    (factored in place): (ranks, rrps, crps[, status])."""
    if not As:
        return ([], [], [], []) if return_status else ([], [], [])
    ctx = ctx or default_context(As[0].device.index)
    b = len(As)
    ms = (ctypes.c_int64 * b)()
    ns = (ctypes.c_int64 * b)()
    lds = (ctypes.c_int64 * b)()
    aptr = (ctypes.c_void_p * b)()
    rptr = (ctypes.c_void_p * b)()
    cptr = (ctypes.c_void_p * b)()
    ranks = (ctypes.c_int64 * b)()
    status = (ctypes.c_int32 * b)()
    R, Cc = [], []
    for i, A in enumerate(As):
        m, n, ld = _matrix_args(A)
        ms[i], ns[i], lds[i] = m, n, ld
        aptr[i] = A.data_ptr() if A.numel() else None
        rr = torch.empty(max(min(m, n), 1), dtype=torch.int32, device=A.device)
        cc = torch.empty(max(min(m, n), 1), dtype=torch.int32, device=A.device)
        R.append(rr)
        Cc.append(cc)
        rptr[i] = rr.data_ptr()
        cptr[i] = cc.data_ptr()
    st = load().rank_profile_modp_batched(ctx.handle, p, b, ms, ns, aptr, lds, rptr, cptr, ranks,
                                          status, _form(form), _stream_handle(stream))
    rk = list(ranks)
    outs = (rk, [R[i][:max(rk[i], 0)] for i in range(b)], [Cc[i][:max(rk[i], 0)] for i in range(b)])
    if return_status:
        return outs + (list(status),)
    _check(st, "rank_profile_modp_batched")
    return outs


def sync_status(ctx: Context) -> int:
    """Waits for the context's stream; the status of its device work (0: OK)."""
    return int(load().pluq_sync_status(ctx.handle))


def last_rank(ctx: Context) -> int:
    r = ctypes.c_int64()
    _check(load().pluq_last_rank(ctx.handle, ctypes.byref(r)), "pluq_last_rank")
    return r.value
