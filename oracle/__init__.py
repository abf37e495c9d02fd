"""CPU oracle for the exact modular matrix multiply on Morton-hybrid matrices.

TEST INFRASTRUCTURE. Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline / reference leg of ``bench.py`` may import or run anything under
``oracle/``. The product library (``paper_1705_04807_gb300``) never imports it,
and this package imports nothing from the product: the two share no code. Their
only common dependency is ``fm_inputs`` (seeded random numbers, no arithmetic of
the method).

What the oracle computes, each part citing the passage it follows:

* ``encode`` / ``extract_i`` / ``extract_j``: the Morton-hybrid index
  (Sec. 1, "Morton-hybrid order"; Sec. 2.2 Step 1 quadrant offsets; Sec. 2.1
  problem P2, in-tile offset ``sigma + i*T' + j``). Written as the quadrant
  recursion in C (``fm_oracle.c``).
* ``to_morton`` / ``from_morton``: layout conversion by that index.
* ``permute``: ``out(i, j) = in(rp[i], cp[j])`` (TURBO's row and column
  permutations, Sec. 1).
* ``gemm_modp``: ``C <- C op A*B mod p`` by the definition (Sec. 2, the
  problem S_A = S_B * S_C over a finite field).
* ``recursion``: the aligned / contained sub-matrix recursion, Steps 1-4 of
  Sec. 2.2, in the paper's notation (module ``oracle.recursion``).
* ``limbs``: residue -> balanced signed 8-bit limbs (module ``oracle.limbs``).
  The paper has no limbs; the reading of the representative is documented there.
* ``pluq``: rank-revealing Gaussian elimination mod p (Sec. 1, TU decomposition
  and rank; the paper defers TURBO's details to its reference, so the textbook
  elimination stands in).
* ``freivalds``: probabilistic check of a product through ``matvec_modp``.
* ``hilbert``: the Hilbert-hybrid layout (the curve Sec. 1 weighs against the
  Morton-hybrid order), built from the curve's recursive definition (module
  ``oracle.hilbert``).
* ``gf2_pack`` / ``gf2_unpack``: the bit-packed Morton-hybrid matrix over GF(2)
  (the field of the experiments, Sec. 2.2 "Performance Analysis", T' = 32): the
  Morton-hybrid element order with 32 consecutive entries per word, entry e of
  the order at bit e % 32 of word e // 32. The product over GF(2) is
  ``gemm_modp`` with p = 2.
"""

from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "fm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

OP_SET, OP_ADD, OP_SUB = 0, 1, 2


def build(force: bool = False) -> str:
    """Compile fm_oracle.c with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-shared", "-fPIC", _SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB_PATH)
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        I32 = ctypes.c_int32
        U32 = ctypes.c_uint32
        U64 = ctypes.c_uint64
        lib.or_encode.argtypes = [I64, I64, I32, I64]
        lib.or_encode.restype = U64
        lib.or_extract_i.argtypes = [U64, I32, I64]
        lib.or_extract_i.restype = I64
        lib.or_extract_j.argtypes = [U64, I32, I64]
        lib.or_extract_j.restype = I64
        lib.or_encode_many.argtypes = [P, P, I64, I32, I64, P]
        lib.or_encode_many.restype = None
        lib.or_extract_many.argtypes = [P, I64, I32, I64, P, P]
        lib.or_extract_many.restype = None
        lib.or_to_morton.argtypes = [P, I64, I64, I64, P, I32, I64]
        lib.or_to_morton.restype = None
        lib.or_from_morton.argtypes = [P, I32, I64, I64, I64, P, I64]
        lib.or_from_morton.restype = None
        lib.or_permute.argtypes = [P, I64, I64, I64, P, P, P, I64]
        lib.or_permute.restype = None
        lib.or_gemm_modp.argtypes = [P, I64, P, I64, P, I64, I64, I64, I64, U32, I32]
        lib.or_gemm_modp.restype = ctypes.c_int
        lib.or_gemm_modp_entries.argtypes = [P, I64, P, I64, P, I64, I64, U32, I32, P, I64, P]
        lib.or_gemm_modp_entries.restype = ctypes.c_int
        lib.or_matvec_modp.argtypes = [P, I64, I64, I64, P, U32, P]
        lib.or_matvec_modp.restype = ctypes.c_int
        lib.or_pluq.argtypes = [P, I64, I64, U32, P, P]
        lib.or_pluq.restype = I64
        lib.or_set_threads.argtypes = [ctypes.c_int]
        lib.or_set_threads.restype = ctypes.c_int
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _u32(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.uint32)


def set_threads(n: int = 0) -> int:
    """Set the OpenMP thread count (0 keeps it); returns the count in use."""
    return int(_load().or_set_threads(int(n)))


# --------------------------------------------------------------------------
# Morton-hybrid index (Sec. 1; Sec. 2.2 Step 1; Sec. 2.1 P2)
# --------------------------------------------------------------------------
def encode(i: int, j: int, m: int, T: int) -> int:
    """Morton-hybrid index of Cartesian (i, j) in a (2^m T') x (2^m T') matrix."""
    return int(_load().or_encode(int(i), int(j), int(m), int(T)))


def extract_i(z: int, m: int, T: int) -> int:
    return int(_load().or_extract_i(int(z), int(m), int(T)))


def extract_j(z: int, m: int, T: int) -> int:
    return int(_load().or_extract_j(int(z), int(m), int(T)))


def encode_many(i, j, m: int, T: int) -> np.ndarray:
    i = np.ascontiguousarray(i, dtype=np.int64)
    j = np.ascontiguousarray(j, dtype=np.int64)
    z = np.empty(i.shape, dtype=np.uint64)
    _load().or_encode_many(_ptr(i), _ptr(j), i.size, int(m), int(T), _ptr(z))
    return z


def extract_many(z, m: int, T: int):
    z = np.ascontiguousarray(z, dtype=np.uint64)
    i = np.empty(z.shape, dtype=np.int64)
    j = np.empty(z.shape, dtype=np.int64)
    _load().or_extract_many(_ptr(z), z.size, int(m), int(T), _ptr(i), _ptr(j))
    return i, j


def to_morton(src: np.ndarray, m: int, T: int) -> np.ndarray:
    """Row-major 2-D array -> flat Morton-hybrid array of (2^m T')^2, zero padded."""
    src = _u32(src)
    rows, cols = src.shape
    n = (1 << m) * T
    if rows > n or cols > n:
        raise ValueError("matrix does not fit the Morton grid")
    dst = np.empty(n * n, dtype=np.uint32)
    _load().or_to_morton(_ptr(src), rows, cols, cols, _ptr(dst), int(m), int(T))
    return dst


def from_morton(src: np.ndarray, m: int, T: int, rows: int, cols: int) -> np.ndarray:
    """Flat Morton-hybrid array -> row-major rows x cols corner."""
    src = _u32(src)
    n = (1 << m) * T
    if src.size != n * n:
        raise ValueError("Morton array has the wrong size")
    dst = np.empty((rows, cols), dtype=np.uint32)
    _load().or_from_morton(_ptr(src), int(m), int(T), rows, cols, _ptr(dst), cols)
    return dst


def gf2_pack(src: np.ndarray, m: int) -> np.ndarray:
    """Row-major 0/1 array (bit 0 of each entry) -> words of the bit-packed
    Morton-hybrid matrix of side 2^m * 32: element e of the Morton-hybrid order
    with T' = 32 is bit e % 32 of word e // 32."""
    flat = to_morton(_u32(src) & 1, m, 32).reshape(-1, 32).astype(np.uint64)
    return (flat << np.arange(32, dtype=np.uint64)).sum(axis=1).astype(np.uint32)


def gf2_unpack(words: np.ndarray, m: int, rows: int, cols: int) -> np.ndarray:
    """Inverse of gf2_pack for the leading rows x cols corner."""
    w = _u32(words).astype(np.uint64).reshape(-1, 1)
    flat = ((w >> np.arange(32, dtype=np.uint64)) & 1).astype(np.uint32).reshape(-1)
    return from_morton(flat, m, 32, rows, cols)


def permute(src: np.ndarray, rp=None, cp=None) -> np.ndarray:
    """out(i, j) = src(rp[i], cp[j]); None means the identity."""
    src = _u32(src)
    rows, cols = src.shape
    rpa = None if rp is None else np.ascontiguousarray(rp, dtype=np.int32)
    cpa = None if cp is None else np.ascontiguousarray(cp, dtype=np.int32)
    out_rows = rows if rpa is None else rpa.size
    out_cols = cols if cpa is None else cpa.size
    dst = np.empty((out_rows, out_cols), dtype=np.uint32)
    _load().or_permute(_ptr(src), cols, out_rows, out_cols,
                       None if rpa is None else _ptr(rpa),
                       None if cpa is None else _ptr(cpa), _ptr(dst), out_cols)
    return dst


# --------------------------------------------------------------------------
# Modular product by definition (Sec. 2)
# --------------------------------------------------------------------------
def gemm_modp(C, A, B, p: int, op: int = OP_SUB) -> np.ndarray:
    """Returns C op A*B mod p (op 0 set, 1 add, 2 subtract) for row-major arrays."""
    A = _u32(A)
    B = _u32(B)
    M, K = A.shape
    K2, N = B.shape
    if K != K2:
        raise ValueError("inner dimensions differ")
    out = np.zeros((M, N), dtype=np.uint32) if C is None else _u32(C).copy()
    if out.shape != (M, N):
        raise ValueError("C has the wrong shape")
    rc = _load().or_gemm_modp(_ptr(A), K, _ptr(B), N, _ptr(out), N, M, N, K, int(p), int(op))
    if rc != 0:
        raise ValueError("bad arguments")
    return out


def gemm_modp_entries(C, A, B, p: int, op: int, ij) -> np.ndarray:
    """Entries at the (i, j) pairs in ``ij`` (shape (n, 2)) of C op A*B mod p."""
    A = _u32(A)
    B = _u32(B)
    M, K = A.shape
    N = B.shape[1]
    ij = np.ascontiguousarray(ij, dtype=np.int64).reshape(-1, 2)
    if C is None:
        C = np.zeros((1, N), dtype=np.uint32)
        ldc = N
    else:
        C = _u32(C)
        ldc = C.shape[1]
    out = np.empty(ij.shape[0], dtype=np.uint32)
    rc = _load().or_gemm_modp_entries(_ptr(A), K, _ptr(B), N, _ptr(C), ldc, K, int(p),
                                      int(op), _ptr(ij), ij.shape[0], _ptr(out))
    if rc != 0:
        raise ValueError("bad arguments")
    return out


def matvec_modp(A, x, p: int) -> np.ndarray:
    A = _u32(A)
    x = _u32(x)
    rows, cols = A.shape
    y = np.empty(rows, dtype=np.uint32)
    _load().or_matvec_modp(_ptr(A), cols, rows, cols, _ptr(x), int(p), _ptr(y))
    return y


def freivalds(C_out, C_in, A, B, p: int, op: int, trials: int = 20, seed: int = 0) -> bool:
    """Freivalds' check that C_out == C_in op A*B mod p: for random x,
    C_out x == C_in x op A (B x) mod p. A wrong C_out passes one trial with
    probability at most 1/p."""
    import fm_inputs
    N = B.shape[1]
    for t in range(trials):
        x = fm_inputs.uniform_residues(seed, N, p, stream=1000 + t)
        lhs = matvec_modp(C_out, x, p).astype(np.int64)
        abx = matvec_modp(A, matvec_modp(B, x, p), p).astype(np.int64)
        if op == OP_SET:
            rhs = abx
        else:
            cx = matvec_modp(C_in, x, p).astype(np.int64)
            rhs = (cx + abx) % p if op == OP_ADD else (cx - abx) % p
        if not np.array_equal(lhs, rhs):
            return False
    return True


# --------------------------------------------------------------------------
# Rank-revealing PLUQ (Sec. 1, TU decomposition and rank)
# --------------------------------------------------------------------------
def pluq(A, p: int):
    """Returns (rp, cp, L, U, r) with A[rp][:, cp] == L @ U mod p, L unit lower
    trapezoidal m x r, U upper trapezoidal r x n, r = rank over GF(p)."""
    a = _u32(A).copy()
    m, n = a.shape
    rp = np.empty(m, dtype=np.int32)
    cp = np.empty(n, dtype=np.int32)
    r = int(_load().or_pluq(_ptr(a), m, n, int(p), _ptr(rp), _ptr(cp)))
    if r < 0:
        raise ValueError("bad arguments")
    L = np.zeros((m, r), dtype=np.uint32)
    U = np.zeros((r, n), dtype=np.uint32)
    for t in range(r):
        L[t, t] = 1
        L[t + 1:, t] = a[t + 1:, t]
        U[t, t:] = a[t, t:]
    return rp, cp, L, U, r
