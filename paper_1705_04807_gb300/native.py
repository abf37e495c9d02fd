"""ctypes binding of libfm (include/fm.h): the same entry points, argument
marshalling only. Every computation runs in the library's CUDA kernels; if the
library is missing this module raises instead of falling back to anything.

Pointers may be given as ints or as objects with ``data_ptr()`` (torch
tensors); streams as ints, ``torch.cuda.Stream`` objects, or None for the
current torch stream (legacy default stream when torch is not loaded).
"""

from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libfm.so")

FM_OK, FM_EINVAL, FM_EMODULUS, FM_ERANGE, FM_ECUDA, FM_ETIMEOUT, FM_ENOMEM, FM_EUNSUPPORTED = (
    0, -1, -2, -3, -4, -5, -6, -7)
FM_ETOOBIG = -8
FM_OP_SET, FM_OP_ADD, FM_OP_SUB = 0, 1, 2
FM_ALGO_AUTO, FM_ALGO_PLAIN, FM_ALGO_LIMB_TC, FM_ALGO_LIMB_MMA_S8, FM_ALGO_DFMA = 0, 1, 2, 3, 4
FM_LIMB_A, FM_LIMB_B = 0, 1
FM_PEAK_IMAD_WIDE, FM_PEAK_IMAD32, FM_PEAK_DFMA, FM_PEAK_FFMA, FM_PEAK_MMA_S8 = 0, 1, 2, 3, 4

# Every symbol include/fm.h declares.
EXPORTS = (
    "fm_layout_to_morton", "fm_layout_to_morton_permuted", "fm_layout_from_morton",
    "fm_layout_to_morton_u16", "fm_layout_to_morton_permuted_u16", "fm_layout_from_morton_u16",
    "fm_validate_residues", "fm_layout_to_hilbert", "fm_layout_from_hilbert", "fm_permute_rows_cols_hilbert",
    "fm_permute_rows_cols", "fm_gemm_modp", "fm_gemm_modp_workspace_size", "fm_plan_create",
    "fm_gemm_modp_batched", "fm_plan_work_items", "fm_plan_launches", "fm_plan_destroy", "fm_decompose",
    "fm_get_last_device_status", "fm_strerror", "fm_release_workspace", "fm_version",
    "fm_limb_planes_size", "fm_limb_split", "fm_limb_gemm", "fm_gemm_modp_noalloc",
    "fm_autotune", "fm_autotune_lookup", "fm_autotune_save", "fm_autotune_load", "fm_autotune_clear",
    "fm_pluq", "fm_gf2_pack", "fm_gf2_unpack", "fm_gf2_gemm", "fm_gf2_workspace_size",
    "fm_gf2_plan_create", "fm_debug_expire_wait", "fm_measure_peak", "fm_autotune_batch",
)


class FmError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        super().__init__(f"{where}: {strerror(code)} ({code})")


class fm_matrix(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("log2_grid", ctypes.c_int32),
                ("log2_T", ctypes.c_int32)]


class fm_sub(ctypes.Structure):
    _fields_ = [("m", fm_matrix), ("row0", ctypes.c_int64), ("col0", ctypes.c_int64),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64)]


class fm_gf2_matrix(ctypes.Structure):
    _fields_ = [("base", ctypes.c_void_p), ("log2_grid", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class fm_gf2_sub(ctypes.Structure):
    _fields_ = [("m", fm_gf2_matrix), ("row0", ctypes.c_int64), ("col0", ctypes.c_int64),
                ("rows", ctypes.c_int64), ("cols", ctypes.c_int64)]


class fm_opts(ctypes.Structure):
    _fields_ = [("k_chunk", ctypes.c_int32), ("block_n", ctypes.c_int32),
                ("no_karatsuba", ctypes.c_int32), ("cta_pair", ctypes.c_int32),
                ("fused_batch", ctypes.c_int32), ("reserved", ctypes.c_int32 * 3)]


class fm_tune_result(ctypes.Structure):
    _fields_ = [("algo", ctypes.c_int32), ("log2_T", ctypes.c_int32), ("opts", fm_opts),
                ("ms", ctypes.c_double), ("gops", ctypes.c_double),
                ("candidates", ctypes.c_int32), ("reserved", ctypes.c_int32)]


FM_TUNE_NO_LIMB, FM_TUNE_NO_PLAIN = 1, 2


class fm_gemm_call(ctypes.Structure):
    _fields_ = [("C", fm_sub), ("A", fm_sub), ("B", fm_sub), ("op", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class fm_gf2_call(ctypes.Structure):
    _fields_ = [("C", fm_gf2_sub), ("A", fm_gf2_sub), ("B", fm_gf2_sub), ("op", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_lib = None


def lib():
    """The loaded libfm (raises ImportError if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libfm.so not found at {LIB_PATH}; build it with "
                          "python -c 'import __graft_entry__ as g; g.build()'")
    L = ctypes.CDLL(LIB_PATH)
    P, I32, I64, U32 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32
    sig = {
        "fm_layout_to_morton": ([P, I64, I64, I64, fm_matrix, P], ctypes.c_int),
        "fm_layout_to_morton_permuted": ([P, I64, I64, I64, P, P, fm_matrix, P], ctypes.c_int),
        "fm_layout_from_morton": ([fm_matrix, I64, I64, P, I64, P], ctypes.c_int),
        "fm_layout_to_morton_u16": ([P, I64, I64, I64, fm_matrix, P], ctypes.c_int),
        "fm_layout_to_morton_permuted_u16": ([P, I64, I64, I64, P, P, fm_matrix, P], ctypes.c_int),
        "fm_layout_from_morton_u16": ([fm_matrix, I64, I64, P, I64, P], ctypes.c_int),
        "fm_validate_residues": ([fm_sub, ctypes.c_uint32, P], ctypes.c_int),
        "fm_layout_to_hilbert": ([P, I64, I64, I64, fm_matrix, P], ctypes.c_int),
        "fm_layout_from_hilbert": ([fm_matrix, I64, I64, P, I64, P], ctypes.c_int),
        "fm_permute_rows_cols_hilbert": ([fm_matrix, fm_matrix, I64, I64, P, P, P], ctypes.c_int),
        "fm_permute_rows_cols": ([fm_matrix, fm_matrix, I64, I64, P, P, P], ctypes.c_int),
        "fm_gemm_modp": ([fm_sub, fm_sub, fm_sub, U32, I32, I32, ctypes.POINTER(fm_opts), P],
                         ctypes.c_int),
        "fm_gemm_modp_workspace_size": ([fm_sub, fm_sub, fm_sub, U32, I32,
                                         ctypes.POINTER(fm_opts)], I64),
        "fm_plan_create": ([ctypes.POINTER(P), ctypes.POINTER(fm_gemm_call), I64, U32, I32,
                            ctypes.POINTER(fm_opts)], ctypes.c_int),
        "fm_gemm_modp_batched": ([P, P], ctypes.c_int),
        "fm_plan_work_items": ([P], I64),
        "fm_plan_launches": ([P], I64),
        "fm_plan_destroy": ([P], ctypes.c_int),
        "fm_decompose": ([fm_sub, fm_sub, fm_sub, ctypes.POINTER(ctypes.c_int64), I64], I64),
        "fm_get_last_device_status": ([P], ctypes.c_int),
        "fm_strerror": ([ctypes.c_int], ctypes.c_char_p),
        "fm_release_workspace": ([], ctypes.c_int),
        "fm_version": ([], ctypes.c_int),
        "fm_limb_planes_size": ([I64, I64, I32, U32, ctypes.POINTER(fm_opts)], I64),
        "fm_limb_split": ([fm_sub, I32, U32, ctypes.POINTER(fm_opts), P, P], ctypes.c_int),
        "fm_limb_gemm": ([fm_sub, P, P, I64, U32, I32, ctypes.POINTER(fm_opts), P], ctypes.c_int),
        "fm_gemm_modp_noalloc": ([fm_sub, fm_sub, fm_sub, U32, I32, P], ctypes.c_int),
        "fm_autotune": ([I64, I64, I64, U32, I32, P, ctypes.POINTER(fm_tune_result)], ctypes.c_int),
        "fm_autotune_lookup": ([I64, I64, I64, U32, ctypes.POINTER(fm_tune_result)], ctypes.c_int),
        "fm_autotune_save": ([ctypes.c_char_p], ctypes.c_int),
        "fm_autotune_load": ([ctypes.c_char_p], ctypes.c_int),
        "fm_autotune_clear": ([], ctypes.c_int),
        "fm_autotune_batch": ([ctypes.POINTER(fm_gemm_call), I64, U32, I32, P, ctypes.POINTER(fm_tune_result)],
                              ctypes.c_int),
        "fm_pluq": ([fm_matrix, I64, I64, U32, P, P, ctypes.POINTER(ctypes.c_int64), P], ctypes.c_int),
        "fm_gf2_pack": ([P, I64, I64, I64, fm_gf2_matrix, P], ctypes.c_int),
        "fm_gf2_unpack": ([fm_gf2_matrix, I64, I64, P, I64, P], ctypes.c_int),
        "fm_gf2_gemm": ([fm_gf2_sub, fm_gf2_sub, fm_gf2_sub, I32, ctypes.POINTER(fm_opts), P],
                        ctypes.c_int),
        "fm_gf2_workspace_size": ([I64, I64, I64], I64),
        "fm_gf2_plan_create": ([ctypes.POINTER(P), ctypes.POINTER(fm_gf2_call), I64,
                                ctypes.POINTER(fm_opts)], ctypes.c_int),
        "fm_debug_expire_wait": ([I32, P], ctypes.c_int),
        "fm_measure_peak": ([I32, I64, P, ctypes.POINTER(ctypes.c_double)], ctypes.c_int),
    }
    for name, (args, res) in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = res
    _lib = L
    return L


def strerror(code: int) -> str:
    try:
        return lib().fm_strerror(int(code)).decode()
    except ImportError:
        return f"status {code}"


def _ptr(x) -> int | None:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    return int(x.data_ptr())


def _stream(s) -> int | None:
    if s is None:
        try:
            import torch
            if torch.cuda.is_available() and torch.cuda.is_initialized():
                return int(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return None
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def _check(rc: int, where: str) -> int:
    if rc != FM_OK:
        raise FmError(rc, where)
    return rc


def matrix(base, log2_grid: int, log2_T: int) -> fm_matrix:
    return fm_matrix(_ptr(base), int(log2_grid), int(log2_T))


def sub(m: fm_matrix, row0: int, col0: int, rows: int, cols: int) -> fm_sub:
    return fm_sub(m, int(row0), int(col0), int(rows), int(cols))


def gf2_matrix(base, log2_grid: int) -> fm_gf2_matrix:
    return fm_gf2_matrix(_ptr(base), int(log2_grid), 0)


def gf2_sub(m: fm_gf2_matrix, row0: int, col0: int, rows: int, cols: int) -> fm_gf2_sub:
    return fm_gf2_sub(m, int(row0), int(col0), int(rows), int(cols))


def opts(k_chunk: int = 0, block_n: int = 0, no_karatsuba: int = 0, cta_pair: int = 0,
         fused_batch: int = 0) -> fm_opts:
    o = fm_opts()
    o.k_chunk = int(k_chunk)
    o.block_n = int(block_n)
    o.no_karatsuba = int(no_karatsuba)
    o.cta_pair = int(cta_pair)
    o.fused_batch = int(fused_batch)
    return o


# ---- entry points (same names as include/fm.h) ----------------------------
def fm_layout_to_morton(src, rows, cols, ld, dst: fm_matrix, stream=None):
    return _check(lib().fm_layout_to_morton(_ptr(src), rows, cols, ld, dst, _stream(stream)),
                  "fm_layout_to_morton")


def fm_layout_to_morton_permuted(src, rows, cols, ld, row_perm, col_perm, dst: fm_matrix,
                                 stream=None):
    return _check(lib().fm_layout_to_morton_permuted(_ptr(src), rows, cols, ld, _ptr(row_perm),
                                                     _ptr(col_perm), dst, _stream(stream)),
                  "fm_layout_to_morton_permuted")


def fm_layout_from_morton(src: fm_matrix, rows, cols, dst, ld, stream=None):
    return _check(lib().fm_layout_from_morton(src, rows, cols, _ptr(dst), ld, _stream(stream)),
                  "fm_layout_from_morton")


def fm_layout_to_morton_u16(src, rows, cols, ld, dst: fm_matrix, stream=None):
    return _check(lib().fm_layout_to_morton_u16(_ptr(src), rows, cols, ld, dst, _stream(stream)),
                  "fm_layout_to_morton_u16")


def fm_layout_to_morton_permuted_u16(src, rows, cols, ld, row_perm, col_perm, dst: fm_matrix,
                                     stream=None):
    return _check(lib().fm_layout_to_morton_permuted_u16(_ptr(src), rows, cols, ld, _ptr(row_perm),
                                                         _ptr(col_perm), dst, _stream(stream)),
                  "fm_layout_to_morton_permuted_u16")


def fm_layout_from_morton_u16(src: fm_matrix, rows, cols, dst, ld, stream=None):
    return _check(lib().fm_layout_from_morton_u16(src, rows, cols, _ptr(dst), ld, _stream(stream)),
                  "fm_layout_from_morton_u16")


def fm_layout_to_hilbert(src, rows, cols, ld, dst: fm_matrix, stream=None):
    return _check(lib().fm_layout_to_hilbert(_ptr(src), rows, cols, ld, dst, _stream(stream)),
                  "fm_layout_to_hilbert")


def fm_layout_from_hilbert(src: fm_matrix, rows, cols, dst, ld, stream=None):
    return _check(lib().fm_layout_from_hilbert(src, rows, cols, _ptr(dst), ld, _stream(stream)),
                  "fm_layout_from_hilbert")


def fm_permute_rows_cols_hilbert(src: fm_matrix, dst: fm_matrix, rows, cols, row_perm, col_perm,
                                 stream=None):
    return _check(lib().fm_permute_rows_cols_hilbert(src, dst, rows, cols, _ptr(row_perm),
                                                     _ptr(col_perm), _stream(stream)),
                  "fm_permute_rows_cols_hilbert")


def fm_validate_residues(X: fm_sub, p: int, stream=None):
    """Checks that every entry of X is below p; a violation shows up as FM_ERANGE
    from fm_get_last_device_status."""
    return _check(lib().fm_validate_residues(X, int(p), _stream(stream)), "fm_validate_residues")


def fm_permute_rows_cols(src: fm_matrix, dst: fm_matrix, rows, cols, row_perm, col_perm,
                         stream=None):
    return _check(lib().fm_permute_rows_cols(src, dst, rows, cols, _ptr(row_perm),
                                             _ptr(col_perm), _stream(stream)),
                  "fm_permute_rows_cols")


def fm_gemm_modp(C: fm_sub, A: fm_sub, B: fm_sub, p: int, op: int = FM_OP_SUB,
                 algo: int = FM_ALGO_AUTO, options: fm_opts | None = None, stream=None):
    o = ctypes.byref(options) if options is not None else None
    return _check(lib().fm_gemm_modp(C, A, B, int(p), int(op), int(algo), o, _stream(stream)),
                  "fm_gemm_modp")


def fm_gemm_modp_noalloc(C: fm_sub, A: fm_sub, B: fm_sub, p: int, op: int = FM_OP_SUB,
                         stream=None):
    """The limb product with no device allocation (fixed 64 MiB scratch; see
    include/fm.h). Raises FmError(FM_ETOOBIG) for larger products."""
    return _check(lib().fm_gemm_modp_noalloc(C, A, B, int(p), int(op), _stream(stream)),
                  "fm_gemm_modp_noalloc")


def fm_gemm_modp_workspace_size(C: fm_sub, A: fm_sub, B: fm_sub, p: int,
                                algo: int = FM_ALGO_AUTO, options: fm_opts | None = None) -> int:
    o = ctypes.byref(options) if options is not None else None
    r = int(lib().fm_gemm_modp_workspace_size(C, A, B, int(p), int(algo), o))
    if r < 0:
        raise FmError(r, "fm_gemm_modp_workspace_size")
    return r


class Plan:
    """Owns an fm_plan (fm_plan_create / fm_plan_destroy)."""

    def __init__(self, calls, p: int, algo: int = FM_ALGO_AUTO, options: fm_opts | None = None,
                 gf2: bool = False):
        h = ctypes.c_void_p()
        o = ctypes.byref(options) if options is not None else None
        if gf2:
            arr = (fm_gf2_call * len(calls))(*calls)
            _check(lib().fm_gf2_plan_create(ctypes.byref(h), arr, len(calls), o), "fm_gf2_plan_create")
        else:
            arr = (fm_gemm_call * len(calls))(*calls)
            _check(lib().fm_plan_create(ctypes.byref(h), arr, len(calls), int(p), int(algo), o),
                   "fm_plan_create")
        self.handle = h

    def run(self, stream=None):
        return fm_gemm_modp_batched(self, stream)

    @property
    def work_items(self) -> int:
        return int(lib().fm_plan_work_items(self.handle))

    @property
    def launches(self) -> int:
        return int(lib().fm_plan_launches(self.handle))

    def close(self):
        if self.handle:
            lib().fm_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def fm_plan_create(calls, p: int, algo: int = FM_ALGO_AUTO, options=None) -> Plan:
    return Plan(calls, p, algo, options)


def fm_gf2_plan_create(calls, options=None) -> Plan:
    """A plan for a batch of GF(2) calls (fm_gf2_call); run it with fm_gemm_modp_batched."""
    return Plan(calls, 2, options=options, gf2=True)


def fm_gemm_modp_batched(plan: Plan, stream=None):
    return _check(lib().fm_gemm_modp_batched(plan.handle, _stream(stream)), "fm_gemm_modp_batched")


def fm_plan_destroy(plan: Plan):
    plan.close()
    return FM_OK


def fm_decompose(C: fm_sub, A: fm_sub, B: fm_sub):
    """Base-case products as a list of (i_lo, i_hi, j_lo, j_hi, l_lo, l_hi)."""
    n = int(lib().fm_decompose(C, A, B, None, 0))
    if n < 0:
        raise FmError(n, "fm_decompose")
    buf = (ctypes.c_int64 * (6 * max(n, 1)))()
    n2 = int(lib().fm_decompose(C, A, B, buf, n))
    return [tuple(buf[6 * t:6 * t + 6]) for t in range(n2)]


def fm_limb_planes_size(rows, cols, role, p, options: fm_opts | None = None) -> int:
    o = ctypes.byref(options) if options is not None else None
    r = int(lib().fm_limb_planes_size(rows, cols, role, int(p), o))
    if r < 0:
        raise FmError(r, "fm_limb_planes_size")
    return r


def fm_limb_split(X: fm_sub, role: int, p: int, planes, options: fm_opts | None = None,
                  stream=None):
    o = ctypes.byref(options) if options is not None else None
    return _check(lib().fm_limb_split(X, int(role), int(p), o, _ptr(planes), _stream(stream)),
                  "fm_limb_split")


def fm_limb_gemm(C: fm_sub, a_planes, b_planes, K: int, p: int, op: int = FM_OP_SUB,
                 options: fm_opts | None = None, stream=None):
    o = ctypes.byref(options) if options is not None else None
    return _check(lib().fm_limb_gemm(C, _ptr(a_planes), _ptr(b_planes), int(K), int(p), int(op),
                                     o, _stream(stream)), "fm_limb_gemm")


def fm_autotune(M: int, N: int, K: int, p: int, flags: int = 0, stream=None) -> fm_tune_result:
    """Times the candidate forms on scratch operands and remembers the fastest."""
    r = fm_tune_result()
    _check(lib().fm_autotune(int(M), int(N), int(K), int(p), int(flags), _stream(stream),
                             ctypes.byref(r)), "fm_autotune")
    return r


def fm_autotune_batch(calls, p: int, flags: int = 0, stream=None) -> fm_tune_result:
    """Times the candidate plan forms on the batch (scratch copies of C) and
    remembers the fastest for its batch class."""
    r = fm_tune_result()
    arr = (fm_gemm_call * len(calls))(*calls)
    _check(lib().fm_autotune_batch(arr, len(calls), int(p), int(flags), _stream(stream), ctypes.byref(r)),
           "fm_autotune_batch")
    return r


def fm_autotune_lookup(M: int, N: int, K: int, p: int):
    r = fm_tune_result()
    hit = int(lib().fm_autotune_lookup(int(M), int(N), int(K), int(p), ctypes.byref(r)))
    if hit < 0:
        raise FmError(hit, "fm_autotune_lookup")
    return r if hit else None


def fm_autotune_save(path: str):
    return _check(lib().fm_autotune_save(os.fsencode(path)), "fm_autotune_save")


def fm_autotune_load(path: str) -> int:
    r = int(lib().fm_autotune_load(os.fsencode(path)))
    if r < 0:
        raise FmError(r, "fm_autotune_load")
    return r


def fm_autotune_clear():
    return _check(lib().fm_autotune_clear(), "fm_autotune_clear")


def fm_pluq(A: fm_matrix, m: int, n: int, p: int, row_perm, col_perm, stream=None) -> int:
    """In-place rank-revealing PLUQ of the leading m x n corner; returns the rank."""
    r = ctypes.c_int64(0)
    _check(lib().fm_pluq(A, int(m), int(n), int(p), _ptr(row_perm), _ptr(col_perm),
                         ctypes.byref(r), _stream(stream)), "fm_pluq")
    return int(r.value)


def fm_gf2_pack(src, rows, cols, ld, dst: fm_gf2_matrix, stream=None):
    return _check(lib().fm_gf2_pack(_ptr(src), rows, cols, ld, dst, _stream(stream)), "fm_gf2_pack")


def fm_gf2_unpack(src: fm_gf2_matrix, rows, cols, dst, ld, stream=None):
    return _check(lib().fm_gf2_unpack(src, rows, cols, _ptr(dst), ld, _stream(stream)),
                  "fm_gf2_unpack")


def fm_gf2_gemm(C: fm_gf2_sub, A: fm_gf2_sub, B: fm_gf2_sub, op: int = FM_OP_SET, options=None,
                stream=None):
    o = ctypes.byref(options) if options is not None else None
    return _check(lib().fm_gf2_gemm(C, A, B, int(op), o, _stream(stream)), "fm_gf2_gemm")


def fm_gf2_workspace_size(M: int, N: int, K: int) -> int:
    r = lib().fm_gf2_workspace_size(int(M), int(N), int(K))
    if r < 0:
        raise FmError(int(r), "fm_gf2_workspace_size")
    return int(r)


def fm_debug_expire_wait(which: int, stream=None):
    return _check(lib().fm_debug_expire_wait(int(which), _stream(stream)), "fm_debug_expire_wait")


def fm_measure_peak(kind: int, iters: int = 1 << 14, stream=None) -> float:
    """Multiply-adds per second of one arithmetic pipe (FM_PEAK_*), measured."""
    out = ctypes.c_double(0.0)
    _check(lib().fm_measure_peak(int(kind), int(iters), _stream(stream), ctypes.byref(out)), "fm_measure_peak")
    return out.value


def fm_get_last_device_status(stream=None) -> int:
    return int(lib().fm_get_last_device_status(_stream(stream)))


def fm_strerror(code: int) -> str:
    return strerror(code)


def fm_release_workspace():
    return _check(lib().fm_release_workspace(), "fm_release_workspace")


def fm_version() -> int:
    return int(lib().fm_version())
