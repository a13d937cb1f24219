"""Python binding of the GB300 CUP library (ctypes over include/cup_gb300.h).

Argument marshalling only: every step of every call runs in the CUDA kernels
of libcup_gb300.so. PyTorch supplies device memory and the current stream.
Residues are held in torch.int32 tensors (values in [0, p) with p < 2^31 are
non-negative, so the bits equal the uint32 the library reads) and index
arrays in torch.int64 tensors. There is no CPU fallback: if the library is
missing or no CUDA device is present, calls raise.
"""
from __future__ import annotations

import ctypes
import os

__all__ = ["load", "Handle", "factor", "rank_profile", "det", "inverse", "rref", "solve",
           "ple", "nullspace", "inplace_mm", "int_det", "int_rank", "crt", "primes_below", "mm_sub", "trsm_ruu", "laswp_cols", "ENGINE_PLAIN", "ENGINE_TENSOR", "CupError",
           "LIB_PATH"]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libcup_gb300.so")
# schedule options measured by tune.py on the GB300, loaded into every handle by default
TUNING_PATH = os.path.join(_HERE, "tuning.json")

ENGINE_PLAIN = 0
ENGINE_TENSOR = 1
OPT_ENGINE, OPT_LEAF_ROWS, OPT_WINDOW, OPT_TC_MIN_K, OPT_VALIDATE, OPT_PROFILE, OPT_SCHEDULE = 0, 1, 2, 3, 4, 5, 6
OPT_INT_PATH = 7
OPT_SHORT_K = 8


class Stats(ctypes.Structure):
    """Mirror of cup_stats (include/cup_gb300.h)."""
    _fields_ = [("launches", ctypes.c_int64), ("host_syncs", ctypes.c_int64),
                ("tc_launches", ctypes.c_int64), ("tc_ms", ctypes.c_double),
                ("tc_limb_flops", ctypes.c_double), ("tc_field_flops", ctypes.c_double),
                ("cc_launches", ctypes.c_int64), ("cc_ms", ctypes.c_double),
                ("cc_field_flops", ctypes.c_double), ("tc_alg_bytes", ctypes.c_double),
                ("sk_launches", ctypes.c_int64), ("sk_ms", ctypes.c_double),
                ("sk_field_flops", ctypes.c_double)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}

STATUS = {0: "CUP_OK", 1: "CUP_SINGULAR", 2: "CUP_INCONSISTENT", -1: "CUP_ERR_ARG",
          -2: "CUP_ERR_PRIME", -3: "CUP_ERR_VALUE", -4: "CUP_ERR_CUDA", -5: "CUP_ERR_TIMEOUT",
          -6: "CUP_ERR_NOMEM", -7: "CUP_ERR_UNSUPPORTED", -8: "CUP_ERR_TOO_LARGE"}

# Every entry point of include/cup_gb300.h with its ctypes signature.
_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_U32 = ctypes.c_uint32
_INT = ctypes.c_int
_I64P = ctypes.POINTER(ctypes.c_int64)
_U32P = ctypes.POINTER(ctypes.c_uint32)
_INTP = ctypes.POINTER(ctypes.c_int)
_DBLP = ctypes.POINTER(ctypes.c_double)
SIGNATURES = {
    "cup_create": (_INT, [ctypes.POINTER(_P), _INT]),
    "cup_destroy": (_INT, [_P]),
    "cup_set_option": (_INT, [_P, _INT, _I64]),
    "cup_last_cuda_error": (ctypes.c_char_p, [_P]),
    "cup_get_stats": (_INT, [_P, _P]),
    "cup_reset_stats": (_INT, [_P]),
    "cup_class_ms": (_INT, [_P, _P]),
    "cup_factor": (_INT, [_P, _P, _I64, _I64, _I64, _U32, _P, _P, _I64P, _P]),
    "cup_factor_host": (_INT, [_P, _P, _I64, _P, _P, _I64, _I64, _I64, _U32, _P, _P, _I64P, _P]),
    "cup_rank_profile": (_INT, [_P, _P, _I64, _I64, _I64, _U32, _P, _I64P, _P]),
    "cup_det": (_INT, [_P, _P, _I64, _I64, _U32, _U32P, _P]),
    "cup_inverse": (_INT, [_P, _P, _I64, _I64, _U32, _P]),
    "cup_rref": (_INT, [_P, _P, _I64, _I64, _I64, _U32, _P, _I64P, _P, _I64, _P]),
    "cup_solve": (_INT, [_P, _P, _I64, _I64, _I64, _P, _I64, _I64, _P, _I64, _U32, _I64P, _P]),
    "cup_nullspace": (_INT, [_P, _P, _I64, _I64, _I64, _U32, _P, _I64, _I64P, _P]),
    "cup_ple": (_INT, [_P, _P, _I64, _I64, _I64, _U32, _P, _P, _I64P, _P]),
    "cup_mm_sub": (_INT, [_P, _P, _I64, _P, _I64, _P, _I64, _I64, _I64, _I64, _U32, _INT, _P]),
    "cup_trsm_ruu": (_INT, [_P, _P, _I64, _P, _I64, _I64, _I64, _U32, _P]),
    "cup_laswp_cols": (_INT, [_P, _P, _I64, _I64, _I64, _P, _I64, _I64, _P]),
    "cup_trsm": (_INT, [_P, _INT, _P, _I64, _P, _I64, _I64, _I64, _U32, _P]),
    "cup_trmm": (_INT, [_P, _INT, _P, _I64, _P, _I64, _I64, _I64, _U32, _P]),
    "cup_trtri": (_INT, [_P, _INT, _P, _I64, _I64, _U32, _P]),
    "cup_trulm": (_INT, [_P, _P, _I64, _I64, _U32, _P]),
    "cup_trlum": (_INT, [_P, _P, _I64, _I64, _U32, _P]),
    "cup_inplace_mm": (_INT, [_P, _P, _I64, _I64, _P, _I64, _I64, _U32, _I64P, _P]),
    "cup_int_bound": (_INT, [_P, _P, _I64, _I64, _I64, _DBLP, _P]),
    "cup_int_det": (_INT, [_P, _P, _I64, _I64, _U32P, _I64, _U32P, _I64, _I64P, _INTP, _I64P, _INTP, _I64P, _P]),
    "cup_int_rank": (_INT, [_P, _P, _I64, _I64, _I64, _U32P, _I64, _I64P, _INTP, _I64P, _P]),
    "cup_crt": (_INT, [_U32P, _U32P, _I64, _U32P, _I64, _I64P, _INTP]),
    "cup_primes_below": (_INT, [_U32, _I64, _U32P, _I64P]),
    "cup_mm_sub_noalloc": (_INT, [_P, _I64, _P, _I64, _P, _I64, _I64, _I64, _I64, _U32, _P]),
    "cup_factor_batched": (_INT, [_P, _P, _I64, _P, _P, _P]),
    "cup_selftest_wait": (_INT, [_P, _I64, _P]),
    "cup_set_tuning": (_INT, [_P, ctypes.c_char_p]),
    "cup_probe_tensor_peak": (_INT, [_INT, _INT, _I64, _DBLP]),
    "cup_factor_u8": (_INT, [_P, _P, _I64, _I64, _I64, _U32, _P, _P, _I64P, _P]),
    "cup_factor_host_u8": (_INT, [_P, _P, _I64, _P, _P, _I64, _I64, _I64, _U32, _P, _P, _I64P, _P]),
    "cup_det_u8": (_INT, [_P, _P, _I64, _I64, _U32, _U32P, _P]),
    "cup_inverse_u8": (_INT, [_P, _P, _I64, _I64, _U32, _P]),
}


class BatchItem(ctypes.Structure):
    """Mirror of cup_batch_item (include/cup_gb300.h)."""
    _fields_ = [("A", ctypes.c_void_p), ("m", ctypes.c_int64), ("n", ctypes.c_int64),
                ("lda", ctypes.c_int64), ("p", ctypes.c_uint32), ("reserved", ctypes.c_uint32),
                ("profile", ctypes.c_void_p), ("ipiv", ctypes.c_void_p)]

LEFT, UPPER, UNIT = 1, 2, 4

_lib = None


class CupError(RuntimeError):
    def __init__(self, status: int, what: str, detail: str = ""):
        self.status = status
        super().__init__(f"{what}: {STATUS.get(status, status)}" + (f" ({detail})" if detail else ""))


def load(path: str | None = None):
    """Load libcup_gb300.so (built by __graft_entry__.build()); raise if absent."""
    global _lib
    if _lib is not None and path is None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"CUDA library {p} is not built; run __graft_entry__.build()")
    lib = ctypes.CDLL(p)
    for name, (res, args) in SIGNATURES.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    if path is None:
        _lib = lib
    return lib


def _torch():
    import torch
    return torch


def _stream_ptr(stream=None):
    torch = _torch()
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _mat(t, what, u8_ok: bool = False):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{what} must be a CUDA tensor")
    if t.dtype not in ((torch.int32, torch.uint8) if u8_ok else (torch.int32,)):
        raise TypeError(f"{what} must be torch.int32 holding residues in [0, p)"
                        + (" (or torch.uint8 for p < 2^8)" if u8_ok else ""))
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{what} must be a row-major 2-D tensor (unit column stride)")
    return t.shape[0], t.shape[1], max(t.stride(0), 1)


def _imat(t, what):
    torch = _torch()
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != torch.int64:
        raise TypeError(f"{what} must be a CUDA torch.int64 tensor of integers")
    if t.dim() != 2 or t.stride(1) != 1:
        raise ValueError(f"{what} must be a row-major 2-D tensor (unit column stride)")
    return t.shape[0], t.shape[1], max(t.stride(0), 1)


def _prime_array(primes):
    if primes is None:
        return None, 0
    arr = (ctypes.c_uint32 * len(primes))(*[int(q) for q in primes])
    return arr, len(primes)


def _from_words(words, nwords: int, sign: int) -> int:
    mag = 0
    for i in range(nwords - 1, -1, -1):
        mag = (mag << 32) | int(words[i])
    return -mag if sign < 0 else mag


class Handle:
    """Owns a cup_handle (and its device workspace) for one CUDA device."""

    def __init__(self, device: int | None = None, engine: int | None = None, tuning=None, **opts):
        """tuning: None loads the tuning table next to the library (if present), a str is a
        table's JSON text or a path to one, False loads none."""
        torch = _torch()
        if not torch.cuda.is_available():
            raise RuntimeError("no CUDA device: the CUP library has no CPU path")
        self.lib = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        self._check(self.lib.cup_create(ctypes.byref(h), self.device), "cup_create", None)
        self.h = h
        if tuning is None and os.path.exists(TUNING_PATH):
            tuning = TUNING_PATH
        if tuning:
            text = open(tuning).read() if os.path.exists(tuning) else tuning
            self._check(self.lib.cup_set_tuning(self.h, text.encode()), "cup_set_tuning", self.h)
        if engine is not None:
            self.set_option(OPT_ENGINE, engine)
        names = {"leaf_rows": OPT_LEAF_ROWS, "window": OPT_WINDOW, "tc_min_k": OPT_TC_MIN_K,
                 "validate": OPT_VALIDATE, "profile": OPT_PROFILE, "schedule": OPT_SCHEDULE,
                 "int_path": OPT_INT_PATH, "short_k": OPT_SHORT_K}
        for k, v in opts.items():
            self.set_option(names[k], int(v))

    def _check(self, st, what, h):
        if st not in (0,):
            detail = ""
            if h is not None and st in (-4, -5):
                detail = self.lib.cup_last_cuda_error(h).decode()
            raise CupError(st, what, detail)

    def set_option(self, opt: int, value: int):
        self._check(self.lib.cup_set_option(self.h, opt, int(value)), "cup_set_option", self.h)

    def stats(self) -> dict:
        st = Stats()
        self._check(self.lib.cup_get_stats(self.h, ctypes.byref(st)), "cup_get_stats", self.h)
        return st.as_dict()

    def class_ms(self) -> dict:
        arr = (ctypes.c_double * 8)()
        self._check(self.lib.cup_class_ms(self.h, arr), "cup_class_ms", self.h)
        names = ["tc_gemm", "cc_gemm", "slab_pivots", "slab_finish", "trsm_leaf", "laswp", "tc_gemm_with_split",
                 "untimed"]
        return {k: arr[i] for i, k in enumerate(names)}

    def reset_stats(self):
        self._check(self.lib.cup_reset_stats(self.h), "cup_reset_stats", self.h)

    def close(self):
        if getattr(self, "h", None):
            self.lib.cup_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def selftest_wait(self, limit_us: int = 200000, stream=None):
        """Run cup_selftest_wait: a device wait that nothing completes, given up after
        limit_us. Returns (status, message); status is -5 (CUP_ERR_TIMEOUT) when the
        bounded wait and its reporting work."""
        st = self.lib.cup_selftest_wait(self.h, int(limit_us), _stream_ptr(stream))
        return st, self.lib.cup_last_cuda_error(self.h).decode()

    # --- entry points -----------------------------------------------------
    def factor(self, A, p: int, stream=None):
        """In-place CUP (Algorithm 6): A <- [C\\U]; returns (rank, profile, ipiv)
        with profile/ipiv int64 device tensors of length min(m, n) (first rank valid).
        A torch.uint8 matrix (p < 2^8) goes through cup_factor_u8."""
        torch = _torch()
        m, n, lda = _mat(A, "A", u8_ok=True)
        k = max(min(m, n), 1)
        prof = torch.empty(k, dtype=torch.int64, device=A.device)
        ipiv = torch.empty(k, dtype=torch.int64, device=A.device)
        r = ctypes.c_int64(0)
        fn = "cup_factor_u8" if A.dtype == torch.uint8 else "cup_factor"
        st = getattr(self.lib, fn)(self.h, A.data_ptr(), m, n, lda, p, prof.data_ptr(),
                                   ipiv.data_ptr(), ctypes.byref(r), _stream_ptr(stream))
        self._check(st, fn, self.h)
        return r.value, prof, ipiv

    def factor_host(self, hA, A, p: int, out=None, stream=None):
        """CUP of a host matrix: hA (CPU int32 tensor, ideally pinned) is copied into the
        device work tensor A in row chunks that overlap the factorization, and [C\\U]
        comes back into `out` (default: hA itself). Returns (rank, profile, ipiv)."""
        torch = _torch()
        dt = A.dtype if isinstance(A, torch.Tensor) else None
        if not isinstance(hA, torch.Tensor) or hA.is_cuda or hA.dtype != dt or hA.dim() != 2 \
                or hA.stride(1) != 1:
            raise TypeError("hA must be a row-major CPU tensor of A's dtype")
        out = hA if out is None else out
        if not isinstance(out, torch.Tensor) or out.is_cuda or out.dtype != dt or out.shape != hA.shape \
                or out.stride() != hA.stride():
            raise TypeError("out must be a CPU tensor laid out like hA")
        m, n, lda = _mat(A, "A", u8_ok=True)
        if tuple(hA.shape) != (m, n):
            raise ValueError("hA and A must have the same shape")
        k = max(min(m, n), 1)
        prof = torch.empty(k, dtype=torch.int64, device=A.device)
        ipiv = torch.empty(k, dtype=torch.int64, device=A.device)
        r = ctypes.c_int64(0)
        fn = "cup_factor_host_u8" if dt == torch.uint8 else "cup_factor_host"
        st = getattr(self.lib, fn)(self.h, hA.data_ptr(), max(hA.stride(0), 1), out.data_ptr(), A.data_ptr(),
                                   m, n, lda, p, prof.data_ptr(), ipiv.data_ptr(), ctypes.byref(r),
                                   _stream_ptr(stream))
        self._check(st, fn, self.h)
        return r.value, prof, ipiv

    def rank_profile(self, A, p: int, stream=None):
        torch = _torch()
        m, n, lda = _mat(A, "A")
        prof = torch.empty(max(min(m, n), 1), dtype=torch.int64, device=A.device)
        r = ctypes.c_int64(0)
        st = self.lib.cup_rank_profile(self.h, A.data_ptr(), m, n, lda, p, prof.data_ptr(),
                                       ctypes.byref(r), _stream_ptr(stream))
        self._check(st, "cup_rank_profile", self.h)
        return r.value, prof[: r.value]

    def det(self, A, p: int, stream=None) -> int:
        torch = _torch()
        n, n2, lda = _mat(A, "A", u8_ok=True)
        if n != n2:
            raise ValueError("det needs a square matrix")
        d = ctypes.c_uint32(0)
        fn = "cup_det_u8" if A.dtype == torch.uint8 else "cup_det"
        st = getattr(self.lib, fn)(self.h, A.data_ptr(), n, lda, p, ctypes.byref(d), _stream_ptr(stream))
        self._check(st, fn, self.h)
        return int(d.value)

    def inverse(self, A, p: int, stream=None) -> bool:
        """A <- A^{-1} in place; returns False (A holds [C\\U]) if A is singular."""
        torch = _torch()
        n, n2, lda = _mat(A, "A", u8_ok=True)
        if n != n2:
            raise ValueError("inverse needs a square matrix")
        fn = "cup_inverse_u8" if A.dtype == torch.uint8 else "cup_inverse"
        st = getattr(self.lib, fn)(self.h, A.data_ptr(), n, lda, p, _stream_ptr(stream))
        if st == 1:
            return False
        self._check(st, fn, self.h)
        return True

    def rref(self, A, p: int, want_x: bool = False, stream=None):
        """A <- R (reduced column echelon form); returns (rank, profile, X or None)."""
        torch = _torch()
        m, n, lda = _mat(A, "A")
        prof = torch.empty(max(min(m, n), 1), dtype=torch.int64, device=A.device)
        X = torch.empty((n, n), dtype=torch.int32, device=A.device) if want_x else None
        r = ctypes.c_int64(0)
        st = self.lib.cup_rref(self.h, A.data_ptr(), m, n, lda, p, prof.data_ptr(), ctypes.byref(r),
                               X.data_ptr() if want_x else None, n if want_x else 0,
                               _stream_ptr(stream))
        self._check(st, "cup_rref", self.h)
        return r.value, prof[: r.value], X

    def ple(self, A, p: int, stream=None):
        """A <- [L\\E] with A = P L E (row echelon twin of CUP); returns (rank, column profile, ipiv)."""
        torch = _torch()
        m, n, lda = _mat(A, "A")
        k = max(min(m, n), 1)
        prof = torch.empty(k, dtype=torch.int64, device=A.device)
        ipiv = torch.empty(k, dtype=torch.int64, device=A.device)
        r = ctypes.c_int64(0)
        st = self.lib.cup_ple(self.h, A.data_ptr(), m, n, lda, p, prof.data_ptr(), ipiv.data_ptr(),
                              ctypes.byref(r), _stream_ptr(stream))
        self._check(st, "cup_ple", self.h)
        return r.value, prof[: r.value], ipiv[: r.value]

    def nullspace(self, A, p: int, stream=None):
        """Basis of {x : A x = 0} (A is destroyed); returns (rank, N) with N of shape (n, n - rank)."""
        torch = _torch()
        m, n, lda = _mat(A, "A")
        Nb = torch.empty((max(n, 1), max(n, 1)), dtype=torch.int32, device=A.device)
        r = ctypes.c_int64(0)
        st = self.lib.cup_nullspace(self.h, A.data_ptr(), m, n, lda, p, Nb.data_ptr(), max(n, 1),
                                    ctypes.byref(r), _stream_ptr(stream))
        self._check(st, "cup_nullspace", self.h)
        return r.value, Nb[:n, : n - r.value]

    def solve(self, A, B, p: int, stream=None):
        """Solve A X = B; returns (status, X, rank) with status 0 or 2 (inconsistent)."""
        torch = _torch()
        m, n, lda = _mat(A, "A")
        mb, k, ldb = _mat(B, "B")
        if mb != m:
            raise ValueError("B must have as many rows as A")
        X = torch.zeros((n, k), dtype=torch.int32, device=A.device)
        r = ctypes.c_int64(0)
        st = self.lib.cup_solve(self.h, A.data_ptr(), m, n, lda, B.data_ptr(), k, ldb,
                                X.data_ptr(), max(k, 1), p, ctypes.byref(r), _stream_ptr(stream))
        if st == 2:
            return 2, X, r.value
        self._check(st, "cup_solve", self.h)
        return 0, X, r.value

    def mm_sub(self, C, A, B, p: int, engine: int = ENGINE_TENSOR, stream=None):
        """C <- C - A B mod p (Algorithm 1 with alpha = -1, beta = 1)."""
        M, N, ldc = _mat(C, "C")
        M2, K, lda = _mat(A, "A")
        K2, N2, ldb = _mat(B, "B")
        if (M2, K2, N2) != (M, K, N):
            raise ValueError("shape mismatch")
        st = self.lib.cup_mm_sub(self.h, C.data_ptr(), ldc, A.data_ptr(), lda, B.data_ptr(), ldb,
                                 M, N, K, p, engine, _stream_ptr(stream))
        self._check(st, "cup_mm_sub", self.h)

    def trsm_ruu(self, U, B, p: int, stream=None):
        """B <- B U^{-1}, U unit upper triangular (strict upper part read)."""
        n, n2, ldu = _mat(U, "U")
        m, nb, ldb = _mat(B, "B")
        if n != n2 or nb != n:
            raise ValueError("shape mismatch")
        st = self.lib.cup_trsm_ruu(self.h, U.data_ptr(), ldu, B.data_ptr(), ldb, m, n, p,
                                   _stream_ptr(stream))
        self._check(st, "cup_trsm_ruu", self.h)

    def trsm(self, flags: int, T, B, p: int, stream=None):
        """B <- T^{-1} B (LEFT) or B T^{-1}; flags from LEFT | UPPER | UNIT."""
        n, n2, ldt = _mat(T, "T")
        rows, cols, ldb = _mat(B, "B")
        if n != n2 or n != (rows if flags & LEFT else cols):
            raise ValueError("shape mismatch")
        st = self.lib.cup_trsm(self.h, flags, T.data_ptr(), ldt, B.data_ptr(), ldb, rows, cols, p,
                               _stream_ptr(stream))
        self._check(st, "cup_trsm", self.h)

    def trmm(self, flags: int, T, B, p: int, stream=None):
        """B <- T B (LEFT) or B T; flags from LEFT | UPPER | UNIT."""
        n, n2, ldt = _mat(T, "T")
        rows, cols, ldb = _mat(B, "B")
        if n != n2 or n != (rows if flags & LEFT else cols):
            raise ValueError("shape mismatch")
        st = self.lib.cup_trmm(self.h, flags, T.data_ptr(), ldt, B.data_ptr(), ldb, rows, cols, p,
                               _stream_ptr(stream))
        self._check(st, "cup_trmm", self.h)

    def trtri(self, flags: int, T, p: int, stream=None):
        n, n2, ldt = _mat(T, "T")
        if n != n2:
            raise ValueError("square triangle needed")
        st = self.lib.cup_trtri(self.h, flags, T.data_ptr(), ldt, n, p, _stream_ptr(stream))
        self._check(st, "cup_trtri", self.h)

    def trulm(self, A, p: int, stream=None):
        n, n2, lda = _mat(A, "A")
        if n != n2:
            raise ValueError("square matrix needed")
        st = self.lib.cup_trulm(self.h, A.data_ptr(), lda, n, p, _stream_ptr(stream))
        self._check(st, "cup_trulm", self.h)

    def trlum(self, A, p: int, stream=None):
        """A = [L\\U] (unit lower L, upper U) <- L U in place."""
        n, n2, lda = _mat(A, "A")
        if n != n2:
            raise ValueError("square matrix needed")
        st = self.lib.cup_trlum(self.h, A.data_ptr(), lda, n, p, _stream_ptr(stream))
        self._check(st, "cup_trlum", self.h)

    def inplace_mm(self, A, B, p: int, stream=None) -> int:
        """B <- A B in place (A square, restored on return); returns rank(A)."""
        m, m2, lda = _mat(A, "A")
        mb, n, ldb = _mat(B, "B")
        if m != m2 or mb != m:
            raise ValueError("A must be m x m and B m x n")
        r = ctypes.c_int64(0)
        st = self.lib.cup_inplace_mm(self.h, A.data_ptr(), m, lda, B.data_ptr(), n, ldb, p,
                                     ctypes.byref(r), _stream_ptr(stream))
        self._check(st, "cup_inplace_mm", self.h)
        return int(r.value)

    def int_bound(self, A, stream=None) -> float:
        """log2 of the product of the nonzero rows' Euclidean norms of an int64 matrix."""
        m, n, lda = _imat(A, "A")
        b = ctypes.c_double(0.0)
        st = self.lib.cup_int_bound(self.h, A.data_ptr(), m, n, lda, ctypes.byref(b), _stream_ptr(stream))
        self._check(st, "cup_int_bound", self.h)
        return float(b.value)

    def int_det(self, A, primes=None, stream=None):
        """det of a square int64 matrix by CUP modulo primes and CRT.
        Returns (det, rank, certified, number of primes used)."""
        n, n2, lda = _imat(A, "A")
        if n != n2:
            raise ValueError("int_det needs a square matrix")
        cap = int(self.int_bound(A, stream) + 33.0) // 32 + 2 if primes is None else len(primes) + 2
        parr, K = _prime_array(primes)
        nw, sg, rk, cert, npr = (ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_int64(0), ctypes.c_int(0),
                                 ctypes.c_int64(0))
        for _ in range(2):
            words = (ctypes.c_uint32 * max(cap, 1))()
            st = self.lib.cup_int_det(self.h, A.data_ptr(), n, lda, parr, K, words, cap, ctypes.byref(nw),
                                      ctypes.byref(sg), ctypes.byref(rk), ctypes.byref(cert), ctypes.byref(npr),
                                      _stream_ptr(stream))
            if st == -8 and nw.value > cap:
                cap = nw.value
                continue
            break
        self._check(st, "cup_int_det", self.h)
        return _from_words(words, nw.value, sg.value), int(rk.value), bool(cert.value), int(npr.value)

    def int_rank(self, A, primes=None, stream=None):
        """rank over Q of an int64 matrix by CUP modulo primes.
        Returns (rank, certified, number of primes used)."""
        m, n, lda = _imat(A, "A")
        parr, K = _prime_array(primes)
        rk, cert, npr = ctypes.c_int64(0), ctypes.c_int(0), ctypes.c_int64(0)
        st = self.lib.cup_int_rank(self.h, A.data_ptr(), m, n, lda, parr, K, ctypes.byref(rk), ctypes.byref(cert),
                                   ctypes.byref(npr), _stream_ptr(stream))
        self._check(st, "cup_int_rank", self.h)
        return int(rk.value), bool(cert.value), int(npr.value)

    def factor_batched(self, mats, primes, want_det: bool = False, stream=None):
        """Batched in-place CUP: mats is a list of int32 CUDA matrices, primes a list of
        primes. Returns (ranks, profiles, ipivs, dets) as device tensors; profile and
        ipiv of matrix b are views of length min(m, n). One launch, no host sync."""
        torch = _torch()
        count = len(mats)
        dev = mats[0].device if count else torch.device("cuda")
        ks = [max(min(t.shape[0], t.shape[1]), 1) for t in mats]
        offs = [0]
        for k in ks:
            offs.append(offs[-1] + k)
        prof = torch.empty(max(offs[-1], 1), dtype=torch.int64, device=dev)
        ipiv = torch.empty(max(offs[-1], 1), dtype=torch.int64, device=dev)
        items = (BatchItem * max(count, 1))()
        for b, (t, p) in enumerate(zip(mats, primes)):
            m, n, lda = _mat(t, "A")
            items[b] = BatchItem(t.data_ptr(), m, n, lda, int(p), 0,
                                 prof.data_ptr() + 8 * offs[b], ipiv.data_ptr() + 8 * offs[b])
        raw = torch.frombuffer(bytearray(items), dtype=torch.uint8)
        d_items = raw.to(dev)
        ranks = torch.empty(max(count, 1), dtype=torch.int64, device=dev)
        dets = torch.empty(max(count, 1), dtype=torch.int32, device=dev) if want_det else None
        st = self.lib.cup_factor_batched(self.h, d_items.data_ptr(), count, ranks.data_ptr(),
                                         dets.data_ptr() if want_det else None, _stream_ptr(stream))
        self._check(st, "cup_factor_batched", self.h)
        self._keep = d_items                     # alive until the stream has used it
        profs = [prof[offs[b]:offs[b] + ks[b]] for b in range(count)]
        ipivs = [ipiv[offs[b]:offs[b] + ks[b]] for b in range(count)]
        return ranks[:count], profs, ipivs, (dets[:count] if want_det else None)

    def laswp_cols(self, A, ipiv, k0: int, k1: int, row0: int = 0, nrows: int | None = None,
                   stream=None):
        m, n, lda = _mat(A, "A")
        nrows = m - row0 if nrows is None else nrows
        st = self.lib.cup_laswp_cols(self.h, A.data_ptr(), lda, row0, nrows, ipiv.data_ptr(),
                                     k0, k1, _stream_ptr(stream))
        self._check(st, "cup_laswp_cols", self.h)


_default = {}


def _handle(engine=None) -> Handle:
    torch = _torch()
    dev = torch.cuda.current_device()
    key = (dev, engine)
    if key not in _default:
        _default[key] = Handle(dev, engine=engine)
    return _default[key]


def factor(A, p, engine=None, stream=None):
    return _handle(engine).factor(A, p, stream)


def rank_profile(A, p, engine=None, stream=None):
    return _handle(engine).rank_profile(A, p, stream)


def det(A, p, engine=None, stream=None):
    return _handle(engine).det(A, p, stream)


def inverse(A, p, engine=None, stream=None):
    return _handle(engine).inverse(A, p, stream)


def rref(A, p, want_x=False, engine=None, stream=None):
    return _handle(engine).rref(A, p, want_x, stream)


def solve(A, B, p, engine=None, stream=None):
    return _handle(engine).solve(A, B, p, stream)


def ple(A, p, engine=None, stream=None):
    return _handle(engine).ple(A, p, stream)


def nullspace(A, p, engine=None, stream=None):
    return _handle(engine).nullspace(A, p, stream)


def inplace_mm(A, B, p, engine=None, stream=None):
    return _handle(engine).inplace_mm(A, B, p, stream)


def int_det(A, primes=None, engine=None, stream=None):
    return _handle(engine).int_det(A, primes, stream)


def int_rank(A, primes=None, engine=None, stream=None):
    return _handle(engine).int_rank(A, primes, stream)


def crt(residues, primes) -> int:
    """The integer in (-M/2, M/2] congruent to residues[i] mod primes[i] (host, no GPU)."""
    lib = load()
    K = len(primes)
    if K != len(residues):
        raise ValueError("one residue per prime")
    r = (ctypes.c_uint32 * K)(*[int(x) for x in residues])
    q = (ctypes.c_uint32 * K)(*[int(x) for x in primes])
    cap = K + 2
    words = (ctypes.c_uint32 * cap)()
    nw, sg = ctypes.c_int64(0), ctypes.c_int(0)
    st = lib.cup_crt(r, q, K, words, cap, ctypes.byref(nw), ctypes.byref(sg))
    if st != 0:
        raise CupError(st, "cup_crt", "")
    return _from_words(words, nw.value, sg.value)


def probe_tensor_peak(kind: int, iters: int | None = None, device: int | None = None) -> float:
    """Measured peak rate (10^12 ops/s) of a tensor instruction on this GPU:
    kind 0 INT8 mma.sync, 1 bf16 mma.sync, 2 tcgen05.mma kind::f16 (cup_probe_tensor_peak)."""
    torch = _torch()
    dev = torch.cuda.current_device() if device is None else int(device)
    iters = iters or (20000 if kind == 2 else 4000)
    out = ctypes.c_double(0.0)
    st = load().cup_probe_tensor_peak(dev, int(kind), int(iters), ctypes.byref(out))
    if st != 0:
        raise CupError(st, "cup_probe_tensor_peak")
    return out.value


def primes_below(bound: int, count: int) -> list:
    """The `count` largest primes below `bound`, descending (host, no GPU)."""
    lib = load()
    out = (ctypes.c_uint32 * max(count, 1))()
    found = ctypes.c_int64(0)
    st = lib.cup_primes_below(int(bound), int(count), out, ctypes.byref(found))
    if st != 0:
        raise CupError(st, "cup_primes_below", "")
    return [int(out[i]) for i in range(found.value)]


def mm_sub(C, A, B, p, engine=ENGINE_TENSOR, stream=None):
    return _handle().mm_sub(C, A, B, p, engine, stream)


def trsm_ruu(U, B, p, stream=None):
    return _handle().trsm_ruu(U, B, p, stream)


def laswp_cols(A, ipiv, k0, k1, row0=0, nrows=None, stream=None):
    return _handle().laswp_cols(A, ipiv, k0, k1, row0, nrows, stream)
