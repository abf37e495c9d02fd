"""GPU parity of the layout and permutation kernels against the oracle (bit-exact)."""
import numpy as np
import pytest

import fm_inputs
from gpu_util import MortonMatrix, lib_and_device, to_dev, to_host

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    return lib_and_device()


@pytest.mark.parametrize("rows,cols,ld,lg,lt", [
    (37, 53, 53, 2, 4), (64, 64, 64, 0, 6), (1, 1, 1, 0, 0), (5, 3, 7, 3, 0), (9, 15, 17, 3, 1),
    (130, 250, 251, 1, 7), (300, 301, 304, 3, 6), (1000, 17, 20, 5, 5), (0, 0, 1, 1, 2)])
def test_to_and_from_morton(env, orc, rows, cols, ld, lg, lt):
    fm, dev = env
    import torch
    x = fm_inputs.uniform_residues(rows * 7 + cols, (rows, ld), 65521)
    M = MortonMatrix(fm, dev, lg, lt)
    M.t.fill_(-1)  # padding must be overwritten with zeros
    fm.fm_layout_to_morton(to_dev(x, dev) if x.size else 0, rows, cols, ld, M.m)
    got = to_host(M.t)
    want = orc.to_morton(x[:, :cols], lg, 1 << lt)
    assert np.array_equal(got, want)
    if rows and cols:
        out = torch.full((rows, ld), -1, dtype=torch.int32, device=dev)
        fm.fm_layout_from_morton(M.m, rows, cols, out, ld)
        back = to_host(out)
        assert np.array_equal(back[:, :cols], x[:, :cols])
        assert np.all(back[:, cols:] == 0xFFFFFFFF)  # columns beyond cols untouched


@pytest.mark.parametrize("rows,cols,lg,lt", [(37, 53, 2, 4), (300, 170, 3, 6), (64, 64, 0, 6)])
def test_to_morton_permuted(env, orc, rows, cols, lg, lt):
    fm, dev = env
    x = fm_inputs.uniform_residues(3, (rows, cols), 65521)
    rp = fm_inputs.permutation(3, rows, 1)
    cp = fm_inputs.permutation(3, cols, 2)
    for r, c in ((rp, cp), (rp, None), (None, cp)):
        M = MortonMatrix(fm, dev, lg, lt)
        fm.fm_layout_to_morton_permuted(to_dev(x, dev), rows, cols, cols,
                                        None if r is None else to_dev(r, dev),
                                        None if c is None else to_dev(c, dev), M.m)
        want = orc.to_morton(orc.permute(x, r, c), lg, 1 << lt)
        assert np.array_equal(to_host(M.t), want)


# (rows, cols, source grid and T', destination grid and T'): T' >= 4 on both
# sides takes the row-staged gather (ragged cols, rows and cols below the
# grid, different T' on the two sides, several tiles), T' < 4 on either side
# the entry-by-entry one
PERMUTE_CASES = [(100, 90, 2, 5, 1, 6), (33, 47, 3, 3, 1, 5), (128, 128, 1, 6, 1, 6),
                 (37, 53, 2, 4, 4, 2), (255, 250, 1, 7, 3, 5), (64, 61, 0, 6, 4, 2),
                 (20, 30, 5, 0, 3, 2), (17, 9, 2, 3, 4, 1), (1, 1, 0, 2, 0, 2), (0, 0, 1, 2, 1, 2)]


@pytest.mark.parametrize("rows,cols,lgs,lts,lgd,ltd", PERMUTE_CASES)
def test_permute_rows_cols(env, orc, rows, cols, lgs, lts, lgd, ltd):
    fm, dev = env
    ns = (1 << lgs) << lts
    x = fm_inputs.uniform_residues(5, (ns, ns), 2147483647)
    S = MortonMatrix(fm, dev, lgs, lts, fill=x)
    nd = (1 << lgd) << ltd
    rp = fm_inputs.permutation(5, rows, 1)
    cp = fm_inputs.permutation(5, cols, 2)
    for r, c in ((rp, cp), (rp, None), (None, cp), (None, None)):
        D = MortonMatrix(fm, dev, lgd, ltd)
        D.t.fill_(-1)  # everything outside rows x cols must become 0
        fm.fm_permute_rows_cols(S.m, D.m, rows, cols, None if r is None or rows == 0 else to_dev(r, dev),
                                None if c is None or cols == 0 else to_dev(c, dev))
        canvas = np.zeros((nd, nd), dtype=np.uint32)
        canvas[:rows, :cols] = orc.permute(x[:rows, :cols], r, c)
        assert np.array_equal(to_host(D.t), orc.to_morton(canvas, lgd, 1 << ltd))
    assert fm.fm_get_last_device_status() == 0


def test_permute_rows_cols_full_size(env, orc):
    # 8192 x 8192 at T' = 32 into T' = 128 (the row-staged gather with 32 KB
    # source rows), every entry compared with the oracle's permutation
    import torch
    fm, dev = env
    n = 8192
    x = fm_inputs.uniform_residues(8, (n, n), 65521)
    rp = fm_inputs.permutation(8, n, 1)
    cp = fm_inputs.permutation(8, n, 2)
    S = MortonMatrix(fm, dev, 8, 5, fill=x)
    D = MortonMatrix(fm, dev, 6, 7)
    fm.fm_permute_rows_cols(S.m, D.m, n, n, to_dev(rp, dev), to_dev(cp, dev))
    got = D.read()
    assert fm.fm_get_last_device_status() == 0
    assert np.array_equal(got, orc.permute(x, rp, cp))
    del S, D
    torch.cuda.empty_cache()


def _bad(perm, where, value):
    out = perm.copy()
    out[where] = value
    return out


@pytest.mark.parametrize("rows,cols,lgs,lts,lgd,ltd", [(100, 90, 2, 5, 1, 6), (37, 53, 2, 4, 4, 2),
                                                        (20, 30, 5, 0, 3, 2)])
def test_permute_out_of_range_entries(env, orc, rows, cols, lgs, lts, lgd, ltd):
    # a permutation entry outside [0, rows) / [0, cols) (too large, or
    # negative) is never used as an index: the entries it would fill are 0,
    # everything else is the permutation, and FM_EINVAL arrives in the status
    fm, dev = env
    ns, nd = (1 << lgs) << lts, (1 << lgd) << ltd
    x = fm_inputs.uniform_residues(6, (ns, ns), 65521)
    S = MortonMatrix(fm, dev, lgs, lts, fill=x)
    rp = fm_inputs.permutation(6, rows, 1)
    cp = fm_inputs.permutation(6, cols, 2)
    assert fm.fm_get_last_device_status() == 0
    for r, c, zero_row, zero_col in ((_bad(rp, 3, rows), cp, 3, None), (_bad(rp, 5, -7), cp, 5, None),
                                     (rp, _bad(cp, 4, cols + 1000), None, 4), (rp, _bad(cp, 2, -1), None, 2),
                                     (None, _bad(cp, cols - 1, 1 << 30), None, cols - 1)):
        D = MortonMatrix(fm, dev, lgd, ltd)
        fm.fm_permute_rows_cols(S.m, D.m, rows, cols, None if r is None else to_dev(r, dev), to_dev(c, dev))
        got = D.read(rows, cols)
        assert fm.fm_get_last_device_status() == fm.FM_EINVAL
        good_r = np.arange(rows) if r is None else np.where((r >= 0) & (r < rows), r, 0)
        good_c = np.where((c >= 0) & (c < cols), c, 0)
        want = orc.permute(x[:rows, :cols], good_r, good_c)
        if zero_row is not None:
            want[zero_row, :] = 0
        if zero_col is not None:
            want[:, zero_col] = 0
        assert np.array_equal(got, want)
    assert fm.fm_get_last_device_status() == 0  # reading cleared it


@pytest.mark.parametrize("rows,cols,lg,lt,u16", [(37, 53, 2, 4, False), (300, 170, 3, 6, True), (9, 15, 3, 1, False)])
def test_to_morton_permuted_out_of_range_entries(env, orc, rows, cols, lg, lt, u16):
    # the same for the row-major -> Morton-hybrid conversion: with a column
    # permutation (the row-staged kernel; T' >= 4), with only a row permutation
    # (the tile walk), and at T' = 2 (entry by entry)
    import torch
    fm, dev = env
    x = fm_inputs.uniform_residues(7, (rows, cols), 65521)
    src = torch.from_numpy(x.astype(np.uint16).view(np.int16)).to(dev) if u16 else to_dev(x, dev)
    conv = fm.fm_layout_to_morton_permuted_u16 if u16 else fm.fm_layout_to_morton_permuted
    rp = fm_inputs.permutation(7, rows, 1)
    cp = fm_inputs.permutation(7, cols, 2)
    assert fm.fm_get_last_device_status() == 0
    for r, c, zero_row, zero_col in ((_bad(rp, 1, rows), cp, 1, None), (_bad(rp, 2, -3), None, 2, None),
                                     (rp, _bad(cp, 6, cols), None, 6), (None, _bad(cp, 0, -100), None, 0)):
        M = MortonMatrix(fm, dev, lg, lt)
        M.t.fill_(-1)
        conv(src, rows, cols, cols, None if r is None else to_dev(r, dev), None if c is None else to_dev(c, dev),
             M.m)
        got = M.read(rows, cols)
        assert fm.fm_get_last_device_status() == fm.FM_EINVAL
        good_r = np.arange(rows) if r is None else np.where((r >= 0) & (r < rows), r, 0)
        good_c = np.arange(cols) if c is None else np.where((c >= 0) & (c < cols), c, 0)
        want = orc.permute(x, good_r, good_c)
        if zero_row is not None:
            want[zero_row, :] = 0
        if zero_col is not None:
            want[:, zero_col] = 0
        assert np.array_equal(got, want)


def test_layout_errors(env):
    fm, dev = env
    M = MortonMatrix(fm, dev, 1, 5)
    import torch
    src = torch.zeros(100 * 100, dtype=torch.int32, device=dev)
    with pytest.raises(fm.FmError):
        fm.fm_layout_to_morton(src, 65, 10, 10, M.m)      # more rows than the grid
    with pytest.raises(fm.FmError):
        fm.fm_layout_to_morton(src, 10, 10, 5, M.m)       # ld < cols
    with pytest.raises(fm.FmError):
        fm.fm_permute_rows_cols(M.m, M.m, 10, 10, None, None)  # src == dst


def test_config2_layout_full_size(env, orc):
    # 3000 x 1700 and 1700 x 2200 row-major residues, random row and column
    # permutations, converted to Morton-hybrid 4096 x 4096 grids at T' = 64.
    fm, dev = env
    p = 65521
    for (rows, cols, seed) in ((3000, 1700, 11), (1700, 2200, 12)):
        x = fm_inputs.uniform_residues(seed, (rows, cols), p)
        rp = fm_inputs.permutation(seed, rows, 1)
        cp = fm_inputs.permutation(seed, cols, 2)
        M = MortonMatrix(fm, dev, 6, 6)
        fm.fm_layout_to_morton_permuted(to_dev(x, dev), rows, cols, cols, to_dev(rp, dev),
                                        to_dev(cp, dev), M.m)
        assert np.array_equal(to_host(M.t), orc.to_morton(orc.permute(x, rp, cp), 6, 64))


@pytest.mark.parametrize("rows,cols,ld,lg,lt", [(37, 53, 53, 2, 4), (300, 301, 304, 3, 6), (130, 250, 251, 1, 7),
                                                (5, 3, 7, 3, 0), (1000, 17, 20, 5, 5), (64, 64, 64, 0, 6)])
def test_u16_layout_matches_u32(env, orc, rows, cols, ld, lg, lt):
    # 16-bit row-major entries (residues mod 65521): the same Morton-hybrid
    # matrix as the 32-bit conversion, with and without permutations, and the
    # 16-bit read-back returns the entries and leaves the columns past cols
    import torch
    fm, dev = env
    x = fm_inputs.uniform_residues(rows + 3 * cols, (rows, ld), 65521)
    x16 = x.astype(np.uint16)
    d16 = torch.from_numpy(x16.view(np.int16)).to(dev)
    M = MortonMatrix(fm, dev, lg, lt)
    M.t.fill_(-1)
    fm.fm_layout_to_morton_u16(d16, rows, cols, ld, M.m)
    assert np.array_equal(to_host(M.t), orc.to_morton(x[:, :cols], lg, 1 << lt))
    out = torch.full((rows, ld), -1, dtype=torch.int16, device=dev)
    fm.fm_layout_from_morton_u16(M.m, rows, cols, out, ld)
    back = out.cpu().numpy().view(np.uint16)
    assert np.array_equal(back[:, :cols], x16[:, :cols])
    assert np.all(back[:, cols:] == 0xFFFF)
    rp = fm_inputs.permutation(rows, rows, 1)
    cp = fm_inputs.permutation(cols, cols, 2)
    for r, c in ((rp, cp), (rp, None), (None, cp)):
        P = MortonMatrix(fm, dev, lg, lt)
        fm.fm_layout_to_morton_permuted_u16(d16, rows, cols, ld, None if r is None else to_dev(r, dev),
                                            None if c is None else to_dev(c, dev), P.m)
        want = orc.to_morton(orc.permute(x[:, :cols], r, c), lg, 1 << lt)
        assert np.array_equal(to_host(P.t), want)


@pytest.mark.parametrize("lt,row0,col0,rows,cols", [(5, 3, 7, 100, 90), (6, 0, 0, 256, 256), (3, 17, 5, 1, 200)])
def test_validate_residues(env, lt, row0, col0, rows, cols):
    # a sub-matrix of residues passes; one entry equal to p inside it raises
    # FM_ERANGE; an out-of-range entry outside the sub-matrix is not its business
    import torch
    fm, dev = env
    p = 65521
    n = 256
    lg = 0
    while (1 << lg) << lt < n:
        lg += 1
    x = fm_inputs.uniform_residues(lt + row0, (n, n), p)
    M = MortonMatrix(fm, dev, lg, lt, fill=x)
    X = M.sub(row0, col0, rows, cols)
    fm.fm_get_last_device_status()
    fm.fm_validate_residues(X, p)
    assert fm.fm_get_last_device_status() == 0
    y = x.copy()
    y[row0 + rows // 2, col0 + cols - 1] = p
    if row0 > 0:
        y[row0 - 1, col0] = 0xFFFFFFFF   # outside the sub-matrix
    M.load(y)
    fm.fm_validate_residues(X, p)
    assert fm.fm_get_last_device_status() == fm.FM_ERANGE
    y[row0 + rows // 2, col0 + cols - 1] = p - 1
    M.load(y)
    fm.fm_validate_residues(X, p)
    assert fm.fm_get_last_device_status() == 0


@pytest.mark.parametrize("rows,cols,ld,lg,lt", [(37, 53, 53, 2, 4), (300, 301, 304, 3, 6), (130, 250, 251, 1, 7),
                                                (5, 3, 7, 3, 0), (64, 64, 64, 0, 6), (200, 100, 100, 5, 3)])
def test_hilbert_layout_matches_oracle(env, orc, rows, cols, ld, lg, lt):
    # the Hilbert-hybrid variant: conversion both ways and the permutation
    # gather against the oracle's curve (built by its recursive definition)
    import torch
    from oracle import hilbert
    fm, dev = env
    x = fm_inputs.uniform_residues(rows * 5 + cols, (rows, ld), 65521)
    H = MortonMatrix(fm, dev, lg, lt)
    H.t.fill_(-1)
    fm.fm_layout_to_hilbert(to_dev(x, dev), rows, cols, ld, H.m)
    assert np.array_equal(to_host(H.t), hilbert.to_hilbert(x[:, :cols], lg, 1 << lt))
    out = torch.full((rows, ld), -1, dtype=torch.int32, device=dev)
    fm.fm_layout_from_hilbert(H.m, rows, cols, out, ld)
    back = to_host(out)
    assert np.array_equal(back[:, :cols], x[:, :cols])
    assert np.all(back[:, cols:] == 0xFFFFFFFF)
    rp = fm_inputs.permutation(lt + 1, rows, 1)
    cp = fm_inputs.permutation(lt + 1, cols, 2)
    D = MortonMatrix(fm, dev, lg, lt)
    D.t.fill_(-1)
    fm.fm_permute_rows_cols_hilbert(H.m, D.m, rows, cols, to_dev(rp, dev), to_dev(cp, dev))
    want = hilbert.to_hilbert(orc.permute(x[:, :cols], rp, cp), lg, 1 << lt)
    assert np.array_equal(to_host(D.t), want)
