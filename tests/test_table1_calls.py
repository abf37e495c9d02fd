"""The call-count column of the paper's Table 1 (Sec. 2.2, "Performance Analysis"),
hardware-independent: for 468 products of random sub-matrices of three
2048 x 2048 Morton-hybrid matrices with T' = 32, the percentage more base-case
calls made by the aligned/contained recursion (Steps 1-4) than by the default
recursion on the sub-matrices' own dimensions.

The aligned count comes from the library's host-only decomposition
(fm_decompose, pinned to the oracle's recursion in test_abi.py and again here
on small cases); the default count from the oracle's default_calls, whose
algorithm the paper does not print (parity unpinned). Run with -s to print the
distribution next to the paper's.

    python -m pytest tests/test_table1_calls.py -s -q
"""
import collections
import functools

import pytest

import fm_inputs

N, T, LT, EXPERIMENTS = 2048, 32, 5, 468

# Table 1 of the paper: % increase in calls -> % of experiments
PAPER = {0: 6.8, 3.13: 1.7, 6.25: 1.7, 24.14: 1.3, 34.38: 9.4, 37.5: 20.3, 38.57: 0.9, 41.8: 0.9,
         42.77: 0.9, 46.09: 0.9, 80.57: 2.6, 84.77: 5.1, 100: 18.6, 106.25: 1.7, 112.5: 1.7,
         168.75: 10.3, 175: 5.1, 300: 10.3}


@pytest.fixture(scope="module")
def fm():
    from paper_1705_04807_gb300 import build
    build.build()
    import paper_1705_04807_gb300 as fm
    fm.lib()
    return fm


def aligned_calls(fm, rect, lg):
    M, N_, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rect)
    mats = [fm.matrix(q << 20, lg, LT) for q in (1, 2, 3)]  # host-only: distinct fake bases
    C = fm.sub(mats[0], rC, cC, M, N_)
    A = fm.sub(mats[1], rA, cA, M, K)
    B = fm.sub(mats[2], rB, cB, K, N_)
    n = int(fm.lib().fm_decompose(C, A, B, None, 0))
    assert n >= 0
    return n


def test_aligned_count_matches_oracle_recursion_on_small_cases(fm):
    from oracle import recursion
    lg = 3  # 256 x 256 matrices, T' = 32
    for rect in fm_inputs.sub_rectangles(11, 40, 256):
        M, N_, K, rC, cC, rA, cA, rB, cB = (int(x) for x in rect)
        want = len(recursion.leaves(lg, T, (rC, cC, M, N_), (rA, cA, M, K), (rB, cB, K, N_)))
        assert aligned_calls(fm, rect, lg) == want


def test_default_calls_special_cases():
    from oracle import recursion
    # one base case at or below T'; a full 2^k T' cube splits into 8^k
    assert recursion.default_calls(T, 32, 32, 32) == 1
    assert recursion.default_calls(T, 64, 64, 64) == 8
    assert recursion.default_calls(T, 2048, 2048, 2048) == 64 ** 3
    assert recursion.default_calls(T, 33, 1, 1) == 2


def _leaves_per_dim(x):
    # Closed form of the halving recursion along one dimension: for
    # 2^k T' < x <= 2^(k+1) T', the pieces at depth k have sizes floor and ceil
    # of x / 2^k (at most 2T'), and each piece longer than T' splits once more;
    # x - 2^k T' of them are longer when that is below 2^k, all 2^k otherwise.
    if x <= T:
        return 1
    k = 0
    while (T << (k + 1)) < x:
        k += 1
    return (1 << k) + min(1 << k, x - (T << k))


def test_default_calls_closed_form():
    # the default recursion halves every dimension above T' independently, so
    # its base-case count is the product of per-dimension leaf counts, each
    # given by the closed form above (checked on every extent up to 2048 and
    # on mixed triples)
    from oracle import recursion
    for x in range(1, 2049):
        assert recursion.default_calls(T, x, 1, 1) == _leaves_per_dim(x), x
    for M, N_, K in fm_inputs.integers(5, 3 * 100, 1, 1024, 3).reshape(100, 3):
        M, N_, K = int(M), int(N_), int(K)
        assert recursion.default_calls(T, M, N_, K) == _leaves_per_dim(M) * _leaves_per_dim(N_) * _leaves_per_dim(K)


def test_table1_call_increase_distribution(fm):
    from oracle import recursion
    dc = functools.lru_cache(maxsize=None)(lambda M, N_, K: recursion.default_calls(T, M, N_, K))
    lg = 6
    inc = []
    for rect in fm_inputs.sub_rectangles(1705, EXPERIMENTS, N):
        M, N_, K = (int(x) for x in rect[:3])
        a, d = aligned_calls(fm, rect, lg), dc(M, N_, K)
        assert a > 0 and d > 0
        inc.append(round(100.0 * (a - d) / d, 2))
    hist = collections.Counter(inc)
    share = lambda lo, hi: 100.0 * sum(1 for x in inc if lo <= x < hi) / len(inc)  # noqa: E731
    print(f"\n{EXPERIMENTS} random sub-matrix products, N = {N}, T' = {T}")
    print("  % increase in calls (aligned over default): share of experiments, this reading | paper")
    for lo, hi in ((-1e9, 0), (0, 0.005), (0.005, 50), (50, 150), (150, 1e9)):
        paper = sum(v for k, v in PAPER.items() if lo <= k < hi)
        print(f"  [{lo:>6}, {hi:>6}): {share(lo, hi):5.1f} %  | {paper:5.1f} %")
    print("  most frequent values:", ", ".join(f"{k:g}% ({100.0 * v / len(inc):.1f}%)"
                                              for k, v in hist.most_common(8)))
    # the aligned recursion pays extra calls on most random products (the
    # paper's point: Table 1 never shows a decrease and mostly large increases)
    assert share(0.005, 1e9) > 50.0
