"""The seeded input generators: determinism, ranges and shape rules."""
import numpy as np

import fm_inputs


def test_splitmix64_published_values():
    # SplitMix64 output function on 0x9E3779B97F4A7C15 * k (state after k steps from
    # seed 0) gives the generator's well-known first outputs for seed 0.
    z = fm_inputs._mix(np.array([0x9E3779B97F4A7C15, 0x3C6EF372FE94F82A], dtype=np.uint64))
    assert int(z[0]) == 0xE220A8397B1DCDAF
    assert int(z[1]) == 0x6E789E6AA1B965F4


def test_residues_deterministic_and_in_range():
    for p in (2, 65521, 2147483647):
        a = fm_inputs.uniform_residues(7, (100, 33), p)
        b = fm_inputs.uniform_residues(7, (100, 33), p)
        assert a.dtype == np.uint32 and a.shape == (100, 33)
        assert np.array_equal(a, b)
        assert a.max() < p
    assert not np.array_equal(fm_inputs.uniform_residues(7, 64, 65521, 0),
                              fm_inputs.uniform_residues(7, 64, 65521, 1))


def test_residues_roughly_uniform():
    p = 17
    x = fm_inputs.uniform_residues(1, 170000, p)
    counts = np.bincount(x, minlength=p)
    assert counts.min() > 9000 and counts.max() < 11000


def test_permutation_and_shapes():
    pr = fm_inputs.permutation(3, 1000)
    assert sorted(pr.tolist()) == list(range(1000))
    s = fm_inputs.batch_shapes(1, 500, 32, 512)
    assert s.shape == (500, 3) and s.min() >= 32 and s.max() <= 512
    r = fm_inputs.sub_rectangles(2, 50, 64)
    M, N, K = r[:, 0], r[:, 1], r[:, 2]
    assert np.all(r[:, 3] + M <= 64) and np.all(r[:, 4] + N <= 64)
    assert np.all(r[:, 5] + M <= 64) and np.all(r[:, 6] + K <= 64)
    assert np.all(r[:, 7] + K <= 64) and np.all(r[:, 8] + N <= 64)


def test_batch_workload_geometry():
    # every call inside its own cell of C and inside the shared A and B
    rows, cells = fm_inputs.batch_workload(5, 300, 32, 512, 4096)
    assert cells == 32 and rows.shape == (300, 9)
    rows2, _ = fm_inputs.batch_workload(5, 300, 32, 512, 4096)
    assert np.array_equal(rows, rows2)
    M, N, K = rows[:, 0], rows[:, 1], rows[:, 2]
    assert M.min() >= 32 and max(M.max(), N.max(), K.max()) <= 512
    c = np.arange(300)
    assert np.array_equal(rows[:, 3], (c // cells) * 512) and np.array_equal(rows[:, 4], (c % cells) * 512)
    assert np.all(rows[:, 5] + M <= 4096) and np.all(rows[:, 6] + K <= 4096)
    assert np.all(rows[:, 7] + K <= 4096) and np.all(rows[:, 8] + N <= 4096)
    assert np.all(rows[:, 5:] >= 0)
