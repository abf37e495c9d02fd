"""Planted mistakes in the oracle: its pins must catch every one (CPU only).

The oracle is pinned to values and properties that the paper and the
mathematics fix (hand-derived tables, brute force, closed forms, invariants),
not to itself. This file checks that those pins are strong enough. For each
oracle function it plants a plausible mistake -- a dropped term, a wrong sign,
a swapped index or bit, a transposed operand, an off-by-one bound -- in a
stand-in for that function (on the CPU; the oracle's files are untouched),
runs the pins of that function against the stand-in, and requires at least
one of them to fail. The same pins run through the same harness against the
real oracle must all pass, so a failure comes from the planted mistake and not
from the harness.
"""
import functools
import inspect

import numpy as np
import pytest

import oracle
from oracle import hilbert, limbs, recursion

import test_oracle_gemm
import test_oracle_gf2
import test_oracle_hilbert
import test_oracle_limbs_pluq
import test_oracle_morton
import test_oracle_recursion
import test_table1_calls

ALL_PINS = (test_oracle_gemm, test_oracle_gf2, test_oracle_hilbert, test_oracle_limbs_pluq,
            test_oracle_morton, test_oracle_recursion, test_table1_calls)


# ---------------------------------------------------------------------------
# harness
# ---------------------------------------------------------------------------
def _pin_calls(mod, fixtures):
    """Every pin (test function) of `mod`, expanded over its parametrize marks,
    given the fixtures in `fixtures`; pins that need another fixture are left
    out."""
    calls = []
    for name, fn in sorted(vars(mod).items()):
        if not name.startswith("test_") or not inspect.isfunction(fn):
            continue
        grid = [{}]
        for mark in getattr(fn, "pytestmark", []):
            if mark.name != "parametrize":
                continue
            names = mark.args[0]
            names = [s.strip() for s in names.split(",")] if isinstance(names, str) else list(names)
            rows = []
            for g in grid:
                for v in mark.args[1]:
                    if hasattr(v, "values") and hasattr(v, "marks"):  # pytest.param
                        vals = tuple(v.values)
                    else:
                        vals = tuple(v) if len(names) > 1 else (v,)
                    rows.append({**g, **dict(zip(names, vals))})
            grid = rows
        params = inspect.signature(fn).parameters
        if any(p not in fixtures and p not in grid[0] for p in params):
            continue
        for g in grid:
            kw = {p: fixtures[p] for p in params if p not in g}
            kw.update(g)
            calls.append((f"{mod.__name__}::{name}{sorted(g.items())}", fn, kw))
    return calls


def _run_pins(mods, orc):
    """Runs the pins of `mods` (the oracle passed as `orc` where a pin takes it);
    returns (names of the pins that failed, number of pins run)."""
    failed, ran = [], 0
    for mod in mods:
        for name, fn, kw in _pin_calls(mod, {"orc": orc}):
            ran += 1
            try:
                fn(**kw)
            except pytest.skip.Exception:
                ran -= 1
            except Exception:  # an assertion, or the stand-in refusing its input
                failed.append(name)
    return failed, ran


class _Oracle:
    """The oracle module with some entry points replaced by stand-ins."""

    def __init__(self, base, **stand_ins):
        self._base = base
        self.__dict__.update(stand_ins)

    def __getattr__(self, name):
        return getattr(self._base, name)


def test_every_pin_passes_on_the_real_oracle(orc):
    failed, ran = _run_pins(ALL_PINS, orc)
    assert ran >= 100, ran  # the harness found the pins
    assert failed == []


# ---------------------------------------------------------------------------
# the modular product C op A*B mod p (Sec. 2)
# ---------------------------------------------------------------------------
def _gemm_with(mistake, real):
    def gemm_modp(C, A, B, p, op=oracle.OP_SUB):
        A = np.asarray(A, dtype=np.uint32)
        B = np.asarray(B, dtype=np.uint32)
        if mistake == "transposed_A" and A.shape[0] == A.shape[1]:
            A = np.ascontiguousarray(A.T)
        if mistake == "dropped_last_inner_term" and A.shape[1] > 1:
            A, B = A[:, :-1], B[:-1, :]
        if mistake == "sum_wraps_at_2^64":
            exact = A.astype(object) @ B.astype(object) if A.shape[1] else np.zeros(
                (A.shape[0], B.shape[1]), dtype=object)
            s = np.array([[(int(v) % (1 << 64)) % p for v in row] for row in exact],
                         dtype=np.int64).reshape(A.shape[0], B.shape[1])
        else:
            s = real(None, A, B, p, 0).astype(np.int64)
        c = np.zeros_like(s) if C is None else np.asarray(C, dtype=np.int64)
        if op == 0:
            out = s
        elif op == 1:
            if mistake == "add_not_reduced":
                out = c + s
            elif mistake == "add_ignores_C":
                out = s
            else:
                out = (c + s) % p
        else:
            out = (s - c) % p if mistake == "sub_reversed" else (c - s) % p
        return out.astype(np.uint32)
    return gemm_modp


GEMM_PINS = (test_oracle_gemm, test_oracle_gf2)


@pytest.mark.parametrize("mistake", ["transposed_A", "dropped_last_inner_term", "sum_wraps_at_2^64",
                                     "add_not_reduced", "add_ignores_C", "sub_reversed"])
def test_gemm_pins_catch(orc, mistake):
    failed, _ = _run_pins(GEMM_PINS, _Oracle(orc, gemm_modp=_gemm_with(mistake, orc.gemm_modp)))
    assert failed, mistake


# ---------------------------------------------------------------------------
# the Morton-hybrid index and layout (Sec. 1; Sec. 2.2 Step 1; Sec. 2.1 P2)
# ---------------------------------------------------------------------------
def _morton_with(mistake):
    def tile_index(I, J, m):
        if mistake == "tiles_in_row_major_order":
            return I * (1 << m) + J
        z = np.zeros_like(I)
        for b in range(m):
            ib, jb = (I >> b) & 1, (J >> b) & 1
            if mistake == "row_bits_on_even_positions":
                z |= (ib << (2 * b)) | (jb << (2 * b + 1))
            else:
                z |= (ib << (2 * b + 1)) | (jb << (2 * b))
        return z

    def enc(i, j, m, T):
        i = np.asarray(i, dtype=np.int64)
        j = np.asarray(j, dtype=np.int64)
        I, u, J, v = i // T, i % T, j // T, j % T
        inner = v * T + u if mistake == "tiles_column_major_inside" else u * T + v
        return tile_index(I, J, m) * T * T + inner

    @functools.lru_cache(maxsize=None)
    def inverse(m, T):
        n = (1 << m) * T
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        inv = np.empty(n * n, dtype=np.int64)
        inv[enc(ii.ravel(), jj.ravel(), m, T)] = np.arange(n * n)
        return inv, n

    def ext(z, m, T):
        inv, n = inverse(m, T)
        k = inv[np.asarray(z, dtype=np.int64)]
        return k // n, k % n

    def grid(m, T):
        n = (1 << m) * T
        ii, jj = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
        return n, enc(ii.ravel(), jj.ravel(), m, T)

    def to_morton(src, m, T):
        src = np.asarray(src, dtype=np.uint32)
        n, z = grid(m, T)
        full = np.zeros((n, n), dtype=np.uint32)
        full[:src.shape[0], :src.shape[1]] = src
        out = np.empty(n * n, dtype=np.uint32)
        out[z] = full.ravel()
        return out

    def from_morton(src, m, T, rows, cols):
        n, z = grid(m, T)
        return np.asarray(src, dtype=np.uint32)[z].reshape(n, n)[:rows, :cols].copy()

    return dict(
        encode=lambda i, j, m, T: int(enc(i, j, m, T)),
        extract_i=lambda z, m, T: int(ext(z, m, T)[0]),
        extract_j=lambda z, m, T: int(ext(z, m, T)[1]),
        encode_many=lambda i, j, m, T: enc(i, j, m, T).astype(np.uint64),
        extract_many=ext,
        to_morton=to_morton,
        from_morton=from_morton,
    )


@pytest.mark.parametrize("mistake", ["row_bits_on_even_positions", "tiles_in_row_major_order",
                                     "tiles_column_major_inside"])
def test_morton_pins_catch(orc, mistake):
    failed, _ = _run_pins((test_oracle_morton,), _Oracle(orc, **_morton_with(mistake)))
    assert failed, mistake


def test_morton_stand_in_without_mistake_passes(orc):
    # the stand-in itself is right when no mistake is planted
    failed, _ = _run_pins((test_oracle_morton,), _Oracle(orc, **_morton_with(None)))
    assert failed == []


def test_gemm_stand_in_without_mistake_passes(orc):
    failed, _ = _run_pins(GEMM_PINS, _Oracle(orc, gemm_modp=_gemm_with(None, orc.gemm_modp)))
    assert failed == []


# ---------------------------------------------------------------------------
# the row / column permutation gather out(i, j) = in(rp[i], cp[j]) (Sec. 1)
# ---------------------------------------------------------------------------
def _permute_with(mistake):
    def permute(src, rp=None, cp=None):
        src = np.asarray(src, dtype=np.uint32)
        rows, cols = src.shape
        rp = np.arange(rows) if rp is None else np.asarray(rp, dtype=np.int64)
        cp = np.arange(cols) if cp is None else np.asarray(cp, dtype=np.int64)
        if mistake == "scatter_instead_of_gather":
            out = np.empty_like(src)
            out[np.ix_(rp, cp)] = src
            return out
        if mistake == "columns_ignored":
            return src[rp, :].copy()
        return src[np.ix_(rp, cp)].copy()
    return permute


@pytest.mark.parametrize("mistake", ["scatter_instead_of_gather", "columns_ignored"])
def test_permute_pins_catch(orc, mistake):
    failed, _ = _run_pins((test_oracle_morton,), _Oracle(orc, permute=_permute_with(mistake)))
    assert failed, mistake


def test_permute_stand_in_without_mistake_passes(orc):
    failed, _ = _run_pins((test_oracle_morton,), _Oracle(orc, permute=_permute_with(None)))
    assert failed == []


# ---------------------------------------------------------------------------
# rank-revealing PLUQ (Sec. 1, the TU decomposition)
# ---------------------------------------------------------------------------
def _pluq_with(mistake, real):
    def pluq(A, p):
        rp, cp, L, U, r = real(A, p)
        L, U = L.copy(), U.copy()
        if mistake == "unit_diagonal_of_L_lost" and r > 0:
            L[r - 1, r - 1] = 2 % p
        elif mistake == "rank_one_short" and r > 0:
            r -= 1
            L, U = L[:, :r].copy(), U[:r, :].copy()
        elif mistake == "row_swaps_not_reported":
            rp = np.arange(len(rp), dtype=rp.dtype)
        elif mistake == "column_order_not_reported":
            cp = np.arange(len(cp), dtype=cp.dtype)
        elif mistake == "last_row_of_U_dropped" and r > 0:
            U[r - 1, :] = 0
        return rp, cp, L, U, r
    return pluq


@pytest.mark.parametrize("mistake", ["unit_diagonal_of_L_lost", "rank_one_short", "row_swaps_not_reported",
                                     "column_order_not_reported", "last_row_of_U_dropped"])
def test_pluq_pins_catch(orc, mistake):
    failed, _ = _run_pins((test_oracle_limbs_pluq,), _Oracle(orc, pluq=_pluq_with(mistake, orc.pluq)))
    assert failed, mistake


# ---------------------------------------------------------------------------
# bit-packed GF(2) matrices (Sec. 2.2's experiments: T' = 32 over GF(2))
# ---------------------------------------------------------------------------
def _gf2_with(mistake, monkeypatch):
    def bits(t):
        return (31 - t) if mistake == "high_bit_first" else t

    def order(src, m):
        if mistake == "tiles_of_16":  # the Morton-hybrid order with T' = 16
            return oracle.to_morton(src, m + 1, 16)
        return oracle.to_morton(src, m, 32)

    def unorder(flat, m, rows, cols):
        if mistake == "tiles_of_16":
            return oracle.from_morton(flat, m + 1, 16, rows, cols)
        return oracle.from_morton(flat, m, 32, rows, cols)

    shifts = np.array([bits(t) for t in range(32)], dtype=np.uint64)

    def gf2_pack(src, m):
        flat = order(np.asarray(src, dtype=np.uint32) & 1, m).reshape(-1, 32).astype(np.uint64)
        return (flat << shifts).sum(axis=1).astype(np.uint32)

    def gf2_unpack(words, m, rows, cols):
        w = np.asarray(words, dtype=np.uint32).astype(np.uint64).reshape(-1, 1)
        return unorder(((w >> shifts) & 1).astype(np.uint32).reshape(-1), m, rows, cols)

    monkeypatch.setattr(oracle, "gf2_pack", gf2_pack)
    monkeypatch.setattr(oracle, "gf2_unpack", gf2_unpack)


@pytest.mark.parametrize("mistake", ["high_bit_first", "tiles_of_16"])
def test_gf2_pack_pins_catch(orc, monkeypatch, mistake):
    _gf2_with(mistake, monkeypatch)
    failed, _ = _run_pins((test_oracle_gf2,), orc)
    assert failed, mistake


def test_gf2_stand_in_without_mistake_passes(orc, monkeypatch):
    _gf2_with(None, monkeypatch)
    failed, _ = _run_pins((test_oracle_gf2,), orc)
    assert failed == []


# ---------------------------------------------------------------------------
# balanced signed 8-bit limbs (the tensor-core form's split)
# ---------------------------------------------------------------------------
def _limbs_with(mistake, monkeypatch):
    real_representative = limbs.representative

    def representative(x, p):
        x = np.asarray(x, dtype=np.int64)
        _, hi = limbs.bounds(limbs.n_limbs(p))
        if mistake == "representative_bound_off_by_one":
            return np.where(x < hi, x, x - p)
        if mistake == "representative_at_half_p":
            return np.where(x <= p // 2, x, x - p)
        return real_representative(x, p)

    def split(x, p):
        w = limbs.n_limbs(p)
        v = representative(x, p).astype(np.int64).copy()
        out = np.empty((w,) + v.shape, dtype=np.int8)
        for t in range(w):
            if mistake == "unbalanced_digits":
                d = v % 256
            else:
                d = ((v + 128) % 256) - 128
            out[t] = d.astype(np.int8)
            v = (v - d) // 256
        if np.any(v != 0):
            raise AssertionError("value outside the balanced range")
        if mistake == "digits_high_first":
            out = out[::-1].copy()
        return out

    monkeypatch.setattr(limbs, "representative", representative)
    monkeypatch.setattr(limbs, "split", split)


LIMB_PINS = (test_oracle_limbs_pluq,)


@pytest.mark.parametrize("mistake", ["representative_bound_off_by_one", "representative_at_half_p",
                                     "unbalanced_digits", "digits_high_first"])
def test_limb_pins_catch(orc, monkeypatch, mistake):
    _limbs_with(mistake, monkeypatch)
    failed, _ = _run_pins(LIMB_PINS, orc)
    assert failed, mistake


def test_limb_stand_in_without_mistake_passes(orc, monkeypatch):
    _limbs_with(None, monkeypatch)
    failed, _ = _run_pins(LIMB_PINS, orc)
    assert failed == []


# ---------------------------------------------------------------------------
# the Hilbert curve of the curve variant (Sec. 1)
# ---------------------------------------------------------------------------
def _hilbert_with(mistake, monkeypatch):
    @functools.lru_cache(maxsize=None)
    def curve(m):
        if m == 0:
            return ((0, 0),)
        prev = curve(m - 1)
        s = 1 << (m - 1)
        if mistake == "first_quadrant_not_transposed":
            first = tuple(prev)
        else:
            first = tuple((j, i) for (i, j) in prev)
        second = tuple((i, j + s) for (i, j) in prev)
        third = tuple((i + s, j + s) for (i, j) in prev)
        if mistake == "last_quadrant_transposed":
            fourth = tuple((j + s, i) for (i, j) in prev)
        else:
            fourth = tuple((s - 1 - j + s, s - 1 - i) for (i, j) in prev)
        if mistake == "quadrants_visited_down_first":  # the transposed curve
            second, fourth = (tuple((i + s, j) for (i, j) in prev),
                              tuple((s - 1 - j, s - 1 - i + s) for (i, j) in prev))
            first = tuple((j, i) for (i, j) in prev)
        return first + second + third + fourth

    monkeypatch.setattr(hilbert, "curve", curve)
    if mistake == "tile_index_transposed":
        real_index_map = hilbert.index_map
        real_from = hilbert.from_hilbert

        def to_hilbert(src, m, T):
            src = np.asarray(src, dtype=np.uint32)
            n = (1 << m) * T
            full = np.zeros((n, n), dtype=np.uint32)
            full[:src.shape[0], :src.shape[1]] = src
            H = real_index_map(m)
            out = np.empty(n * n, dtype=np.uint32)
            for I in range(1 << m):
                for J in range(1 << m):
                    base = int(H[J, I]) * T * T
                    out[base:base + T * T] = full[I * T:(I + 1) * T, J * T:(J + 1) * T].reshape(-1)
            return out

        monkeypatch.setattr(hilbert, "to_hilbert", to_hilbert)
        monkeypatch.setattr(hilbert, "from_hilbert", real_from)


@pytest.mark.parametrize("mistake", ["first_quadrant_not_transposed", "last_quadrant_transposed",
                                     "quadrants_visited_down_first", "tile_index_transposed"])
def test_hilbert_pins_catch(orc, monkeypatch, mistake):
    _hilbert_with(mistake, monkeypatch)
    failed, _ = _run_pins((test_oracle_hilbert,), orc)
    assert failed, mistake


def test_hilbert_stand_in_without_mistake_passes(orc, monkeypatch):
    _hilbert_with(None, monkeypatch)
    failed, _ = _run_pins((test_oracle_hilbert,), orc)
    assert failed == []


# ---------------------------------------------------------------------------
# the aligned / contained recursion (Sec. 2.2, Steps 1-4) and the default count
# ---------------------------------------------------------------------------
def _step2_with(mistake, monkeypatch):
    def step2_split(alpha, lam, S, m, T):
        lam_q = lam // 4
        e_NE = alpha + 2 * lam_q - (0 if mistake == "NE_end_off_by_one" else 1)
        e_SW = alpha + 3 * lam_q - 1
        i_S = recursion.extract_i(S.sigma, m, T)
        j_S = recursion.extract_j(S.sigma, m, T)
        r_N = recursion.extract_i(e_NE, m, T) - i_S + 1
        c_W = recursion.extract_j(e_SW, m, T) - j_S + 1
        if mistake != "no_clamp":
            r_N = min(max(r_N, 0), S.r)
            c_W = min(max(c_W, 0), S.c)
        r_S, c_E = S.r - r_N, S.c - c_W
        parts = [recursion._part(i_S, j_S, r_N, c_W, m, T),
                 recursion._part(i_S, j_S + c_W, r_N, c_E, m, T),
                 recursion._part(i_S + r_N, j_S, r_S, c_W, m, T),
                 recursion._part(i_S + r_N, j_S + c_W, r_S, c_E, m, T)]
        if mistake == "NE_and_SW_swapped":
            parts[1], parts[2] = parts[2], parts[1]
        return parts

    monkeypatch.setattr(recursion, "step2_split", step2_split)


RECURSION_PINS = (test_oracle_recursion,)


@pytest.mark.parametrize("mistake", ["NE_end_off_by_one", "no_clamp", "NE_and_SW_swapped"])
def test_recursion_pins_catch(orc, monkeypatch, mistake):
    _step2_with(mistake, monkeypatch)
    failed, _ = _run_pins(RECURSION_PINS, orc)
    assert failed, mistake


def test_recursion_stand_in_without_mistake_passes(orc, monkeypatch):
    _step2_with(None, monkeypatch)
    failed, _ = _run_pins(RECURSION_PINS, orc)
    assert failed == []


def _default_calls_with(mistake):
    def default_calls(T, M, N, K):
        if M == 0 or N == 0 or K == 0:
            return 0
        if mistake == "base_case_checks_M_only":
            if M <= T:
                return 1
        elif M <= T and N <= T and K <= T:
            return 1

        def halves(x):
            if x <= T:
                return [x]
            return [(x + 1) // 2, (x + 1) // 2] if mistake == "both_halves_rounded_up" else [(x + 1) // 2, x // 2]

        return sum(default_calls(T, a, b, c) for a in halves(M) for b in halves(N) for c in halves(K))
    return functools.lru_cache(maxsize=None)(default_calls)


@pytest.mark.parametrize("mistake", ["base_case_checks_M_only", "both_halves_rounded_up"])
def test_default_calls_pins_catch(orc, monkeypatch, mistake):
    monkeypatch.setattr(recursion, "default_calls", _default_calls_with(mistake))
    failed, _ = _run_pins((test_table1_calls, test_oracle_recursion), orc)
    assert failed, mistake


def test_default_calls_stand_in_without_mistake_passes(orc, monkeypatch):
    monkeypatch.setattr(recursion, "default_calls", _default_calls_with(None))
    failed, _ = _run_pins((test_table1_calls, test_oracle_recursion), orc)
    assert failed == []


# ---------------------------------------------------------------------------
# sampled entries and the matrix-vector product behind Freivalds' check
# ---------------------------------------------------------------------------
def _entries_with_swapped_index(real):
    def gemm_modp_entries(C, A, B, p, op, ij):
        ij = np.asarray(ij, dtype=np.int64).reshape(-1, 2)
        full = real(C, A, B, p, op)
        i, j = ij[:, 0], ij[:, 1]
        ok = (j < full.shape[0]) & (i < full.shape[1])
        out = full[i, j].copy()
        out[ok] = full[j[ok], i[ok]]
        return out
    return gemm_modp_entries


def _matvec_dropping_last_term(A, x, p):
    A = np.asarray(A, dtype=np.uint64)
    x = np.asarray(x, dtype=np.uint64)
    if A.shape[1] < 2:
        return (A.astype(object) @ x.astype(object) % p).astype(np.uint32)
    return (A[:, :-1].astype(object) @ x[:-1].astype(object) % p).astype(np.uint32)


def test_entries_pin_catches_a_swapped_index(orc):
    stand_in = _Oracle(orc, gemm_modp_entries=_entries_with_swapped_index(orc.gemm_modp))
    failed, _ = _run_pins((test_oracle_gemm,), stand_in)
    assert failed


def test_freivalds_pin_catches_a_matvec_that_drops_a_term(orc, monkeypatch):
    monkeypatch.setattr(oracle, "matvec_modp", _matvec_dropping_last_term)
    failed, _ = _run_pins((test_oracle_gemm,), orc)
    assert failed
