"""The C ABI: the library loads, exports every symbol include/fm.h declares, and
its host-only decomposition (Sec. 2.2) matches the oracle's recursion. No GPU."""
import os
import re

import pytest

from conftest import ROOT

import fm_inputs


@pytest.fixture(scope="module")
def fm():
    import __graft_entry__
    from paper_1705_04807_gb300 import build
    build.build()
    import paper_1705_04807_gb300 as fm
    fm.lib()
    return fm


def declared_functions():
    names = set()
    inc = os.path.join(ROOT, "include")
    for f in os.listdir(inc):
        if not f.endswith(".h"):
            continue
        text = open(os.path.join(inc, f)).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(fm_\w+)\s*\(", text, re.M):
            names.add(m.group(1))
    return names


def test_exports_every_declared_symbol(fm):
    declared = declared_functions()
    assert {"fm_gemm_modp", "fm_layout_to_morton", "fm_layout_from_morton",
            "fm_permute_rows_cols", "fm_gemm_modp_batched"} <= declared
    lib = fm.lib()
    for name in declared:
        assert hasattr(lib, name), name
    assert declared == set(fm.EXPORTS)


def test_version_and_strerror(fm):
    assert fm.fm_version() == 100
    assert "modulus" in fm.fm_strerror(fm.FM_EMODULUS)
    assert fm.fm_strerror(0) == "ok"


def _subs(fm, n_lg, lt, rect):
    M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rect)
    fake = 1 << 20  # host-only call: any aligned non-null base, distinct per matrix
    mC, mA, mB = fm.matrix(fake, n_lg, lt), fm.matrix(2 * fake, n_lg, lt), fm.matrix(3 * fake, n_lg, lt)
    return fm.sub(mC, rC, cC, M, N), fm.sub(mA, rA, cA, M, K), fm.sub(mB, rB, cB, K, N)


@pytest.mark.parametrize("lg,lt", [(2, 1), (3, 1), (2, 2), (1, 3)])
def test_decomposition_matches_oracle_recursion(fm, lg, lt):
    from oracle import recursion
    T = 1 << lt
    n = (1 << lg) * T
    for rect in fm_inputs.sub_rectangles(lg * 7 + lt, 20, n):
        C, A, B = _subs(fm, lg, lt, rect)
        got = sorted(fm.fm_decompose(C, A, B))
        M, N, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rect)
        # paper naming: S_A (output) = C, S_B = A, S_C = B
        leaves = recursion.leaves(lg, T, (rC, cC, M, N), (rA, cA, M, K), (rB, cB, K, N))
        want = sorted((l.i_lo, l.i_hi, l.j_lo, l.j_hi, l.l_lo, l.l_hi) for l in leaves)
        assert got == want


def test_decompose_rejects_bad_operands(fm):
    mC, mA = fm.matrix(1 << 20, 2, 5), fm.matrix(2 << 20, 2, 5)
    with pytest.raises(fm.FmError):
        fm.fm_decompose(fm.sub(mC, 0, 0, 10, 10), fm.sub(mA, 0, 0, 11, 4), fm.sub(mA, 0, 0, 4, 10))
    with pytest.raises(fm.FmError):   # outside the matrix
        fm.fm_decompose(fm.sub(mC, 120, 0, 10, 10), fm.sub(mA, 0, 0, 10, 4), fm.sub(mA, 0, 0, 4, 10))
    with pytest.raises(fm.FmError):   # C overlaps A
        fm.fm_decompose(fm.sub(mC, 0, 0, 10, 10), fm.sub(mC, 5, 5, 10, 4), fm.sub(mA, 0, 0, 4, 10))
    with pytest.raises(fm.FmError):   # different T'
        fm.fm_decompose(fm.sub(mC, 0, 0, 10, 10), fm.sub(fm.matrix(2 << 20, 3, 4), 0, 0, 10, 4),
                        fm.sub(mA, 0, 0, 4, 10))


def test_aligned_decomposition_is_one_product_per_tile_triple(fm):
    C, A, B = _subs(fm, 3, 5, (128, 64, 96, 32, 64, 0, 32, 64, 0))
    assert len(fm.fm_decompose(C, A, B)) == (128 // 32) * (64 // 32) * (96 // 32)


def test_autotune_table_roundtrip(fm, tmp_path):
    # host only: a saved table loads back, drives lookups, and malformed input is refused
    fm.fm_autotune_clear()
    assert fm.fm_autotune_lookup(8192, 8192, 8192, 65521) is None
    table = tmp_path / "tune.txt"
    table.write_text("# libfm autotune table v1\n"
                     "13 13 13 1 2 7 256 960 0 2.500000 439804.651\n"
                     "9 9 9 2 1 6 0 0 0 0.800000 335.544\n")
    assert fm.fm_autotune_load(str(table)) == 2
    r = fm.fm_autotune_lookup(8000, 5000, 4097, 65521)     # rounds up to 2^13 each
    assert r is not None and r.algo == fm.FM_ALGO_LIMB_TC and r.opts.block_n == 256
    assert r.opts.k_chunk == 960 and abs(r.ms - 2.5) < 1e-9
    r2 = fm.fm_autotune_lookup(300, 400, 500, 2147483647)
    assert r2 is not None and r2.algo == fm.FM_ALGO_PLAIN and r2.log2_T == 6
    assert fm.fm_autotune_lookup(300, 400, 500, 65521) is None  # other modulus class
    out = tmp_path / "tune2.txt"
    fm.fm_autotune_save(str(out))
    fm.fm_autotune_clear()
    assert fm.fm_autotune_load(str(out)) == 2
    bad = tmp_path / "bad.txt"
    bad.write_text("1 2 3\n")
    with pytest.raises(fm.FmError):
        fm.fm_autotune_load(str(bad))
    fm.fm_autotune_clear()


def test_autotune_table_batch_lines_roundtrip(fm, tmp_path):
    # host only: batch classes (calls, mean M, N, K, modulus class, T') save and
    # load with the single-call classes; a malformed batch line is refused
    fm.fm_autotune_clear()
    table = tmp_path / "tune.txt"
    table.write_text("# libfm autotune table v2\n"
                     "13 13 13 1 2 7 256 960 0 2.500000 439804.651 1\n"
                     "batch 12 9 9 9 1 6 2 128 960 0 0 4.780000 35100.000\n"
                     "batch 6 5 5 5 2 5 1 0 0 0 0 0.300000 1000.000\n")
    assert fm.fm_autotune_load(str(table)) == 3
    out = tmp_path / "tune2.txt"
    fm.fm_autotune_save(str(out))
    lines = [x for x in out.read_text().splitlines() if x.startswith("batch ")]
    assert lines == ["batch 6 5 5 5 2 5 1 0 0 0 0 0.300000 1000.000",
                     "batch 12 9 9 9 1 6 2 128 960 0 0 4.780000 35100.000"]
    fm.fm_autotune_clear()
    assert fm.fm_autotune_load(str(out)) == 3
    bad = tmp_path / "bad.txt"
    bad.write_text("batch 12 9 9 9 1 6 3 128 960 0 0 4.78 35100\n")  # algo 3 is not a batch form
    with pytest.raises(fm.FmError):
        fm.fm_autotune_load(str(bad))
    fm.fm_autotune_clear()


def test_layout_calls_reject_bad_arguments_on_the_host(fm):
    # argument checks of the 32-bit and 16-bit layout calls run on the host,
    # before any device work (the matrices here are host-only fake bases)
    M = fm.matrix(1 << 20, 1, 5)   # 64 x 64 grid
    for to_morton, from_morton in ((fm.fm_layout_to_morton, fm.fm_layout_from_morton),
                                   (fm.fm_layout_to_morton_u16, fm.fm_layout_from_morton_u16)):
        with pytest.raises(fm.FmError):
            to_morton(1 << 24, 65, 10, 10, M)      # more rows than the grid
        with pytest.raises(fm.FmError):
            to_morton(1 << 24, 10, 10, 5, M)       # ld < cols
        with pytest.raises(fm.FmError):
            to_morton(0, 10, 10, 10, M)            # no source
        with pytest.raises(fm.FmError):
            from_morton(M, 10, 70, 1 << 24, 70)    # more columns than the grid
        with pytest.raises(fm.FmError):
            from_morton(M, 10, 10, 0, 10)          # no destination
    with pytest.raises(fm.FmError):
        fm.fm_layout_to_morton_permuted_u16(1 << 24, 10, 10, 8, 0, 0, M)   # ld < cols


def test_validate_residues_rejects_bad_arguments_on_the_host(fm):
    M = fm.matrix(1 << 20, 1, 5)   # 64 x 64 grid, host-only fake base
    for p in (0, 1, 1 << 31):
        with pytest.raises(fm.FmError):
            fm.fm_validate_residues(fm.sub(M, 0, 0, 8, 8), p)
    with pytest.raises(fm.FmError):
        fm.fm_validate_residues(fm.sub(M, 60, 0, 8, 8), 65521)   # outside the matrix


def test_default_tile_width_follows_the_shape(fm):
    # fm_gemm_modp's limb form sizes its workspace for the planes of the output
    # tile width it will run (host only: without a GPU the SM count takes its
    # default). Fold form: 128-wide tiles for K <= 1024 and for thin products,
    # 256-wide ones for long products with many tiles; an explicit width is
    # kept; the residue form always takes 128.
    lt, lg = 7, 7  # 16384 x 16384 grids at T' = 128; fake bases 4 GiB apart
    C, A, B = (fm.matrix(q << 32, lg, lt) for q in (1, 2, 3))

    def ws(p, M, N, K, o=None):
        return fm.fm_gemm_modp_workspace_size(fm.sub(C, 0, 0, M, N), fm.sub(A, 0, 0, M, K),
                                              fm.sub(B, 0, 0, K, N), p, fm.FM_ALGO_LIMB_TC, o)

    def planes(p, M, N, K, bn):
        o = fm.opts(0, bn)
        return fm.fm_limb_planes_size(M, K, fm.FM_LIMB_A, p, o) + fm.fm_limb_planes_size(K, N, fm.FM_LIMB_B, p, o)

    p16, p31 = 65521, 2147483647
    # shapes whose planes differ between the widths (row blocks padded to an even
    # count at 256, columns to 128 or 256)
    cases = [((8000, 8000, 512), 128),     # short K
             ((8000, 8000, 8192), 256),    # long, many tiles
             ((16000, 100, 2048), 128),    # one column of tiles
             ((100, 11000, 2048), 128)]    # one row block
    for (M, N, K), bn in cases:
        assert planes(p16, M, N, K, 128) != planes(p16, M, N, K, 256)
        assert ws(p16, M, N, K) == planes(p16, M, N, K, bn), (M, N, K)
    assert ws(p16, 8000, 8000, 8192, fm.opts(0, 128)) == planes(p16, 8000, 8000, 8192, 128)
    assert ws(p16, 8000, 8000, 512, fm.opts(0, 256)) == planes(p16, 8000, 8000, 512, 256)
    assert ws(p31, 4000, 4000, 4096) == planes(p31, 4000, 4000, 4096, 128)


def test_limb_planes_size_follows_the_documented_layout(fm):
    # host-only: the plane bytes fm_limb_planes_size reports are the layout the
    # header documents -- per plane, A in ceil(M/128) x ceil(K/64) tiles of
    # 16 KB (row blocks rounded up to even for 256-wide tiles and in the
    # residue form), B in ceil(N/BN) x ceil(K/64) tiles of BN * 128 bytes;
    # planes: 2 limbs + Karatsuba sum (odd p < 2^16), w + w(w-1)/2 (residue
    # form, w limbs and every pair sum), w without Karatsuba
    def cdiv(a, b):
        return -(-a // b)

    cases = [(65521, 3, 256, True), (257, 3, 256, True), (65534, 3, 128, True),
             (65537, 6, 128, True), (2147483647, 10, 128, True)]
    for p, planes, bn, even in cases:
        for M, K, N in ((100, 64, 100), (129, 65, 300), (300, 1000, 129), (1, 1, 1), (4096, 4096, 4096)):
            mb = cdiv(M, 128)
            mb += mb % 2 if even else 0
            kb = cdiv(K, 64)
            assert fm.fm_limb_planes_size(M, K, fm.FM_LIMB_A, p, None) == planes * mb * kb * 16384, (p, M, K)
            assert fm.fm_limb_planes_size(K, N, fm.FM_LIMB_B, p, None) == planes * cdiv(N, bn) * kb * bn * 128, (p, K, N)
    # without Karatsuba the two-limb fold form keeps just its two digit planes
    assert fm.fm_limb_planes_size(100, 64, fm.FM_LIMB_A, 65521, fm.opts(no_karatsuba=1)) == 2 * 2 * 1 * 16384
    for bad in ((-1, 64, fm.FM_LIMB_A, 65521), (64, 64, 7, 65521), (64, 64, fm.FM_LIMB_A, 1)):
        with pytest.raises(fm.FmError):
            fm.fm_limb_planes_size(*bad)
