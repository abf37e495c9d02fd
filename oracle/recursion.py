"""The aligned / contained sub-matrix recursion of Sec. 2.2, in the paper's notation.

TEST INFRASTRUCTURE (see ``oracle/__init__.py``).

The paper multiplies sub-matrices S_A = S_B * S_C of Morton-hybrid matrices A,
B, C of equal size (2^m T') x (2^m T'). Instead of dividing the sub-matrices,
it divides the aligned parents A^k, B^k, C^k, each identified by
(alpha, lambda) = (Morton index of the first entry, number of entries), and
carries along the part S of the sub-matrix inside each, identified by the
4-tuple (M, sigma, r, c) (Sec. 2.2, definitions after the Step-list intro).

Step 1: quadrant q of an aligned block starts at alpha + q*lambda', with
        lambda' = lambda / 4 and the order NW=0, NE=1, SW=2, SE=3.
Step 2: e_NE = alpha + 2 lambda' - 1, e_SW = alpha + 3 lambda' - 1;
        r_N = extract_i(e_NE) - extract_i(sigma_S) + 1,
        c_W = extract_j(e_SW) - extract_j(sigma_S) + 1,
        r_S = r - r_N, c_E = c - c_W; the four parts S' follow with
        encode(i_S + {0, r_N}, j_S + {0, c_W}).
Step 3: all 4 x 4 x 4 = 64 combinations of quadrants of A, B and C.
Step 4: keep the compatible parts of each combination and recurse.

Readings taken where the text is silent, garbled or inconsistent:

* c_W is printed with alpha_S; it is read as sigma_S (the first entry of S),
  matching r_N's formula.
* r_N and c_W are clamped to [0, r] and [0, c]: the text says only that a
  value <= 0 means no part in that half; a value above r (S entirely in the
  north half) means all of it.
* The fourth part is printed twice as S'_SW; the second one is S'_SE.
* Step 4 ("extract compatible parts") is left unspecified by the paper. Reading:
  the product S_A += S_B * S_C has three local index ranges, output row i,
  output column j and inner index l; row i is row i_A + i of A and row i_B + i
  of B, column j is column j_A + j of A and column j_C + j of C, inner l is
  column j_B + l of B and row i_C + l of C. A part of A restricts (i, j), a
  part of B restricts (i, l), a part of C restricts (l, j). A combination is
  compatible on the intersections of these ranges, and proceeds on those
  intersections when all three are non-empty.

The base case (lambda = T'^2) emits one triple of contained parts. This module
returns those triples; tests check them against brute force and the paper's
propositions (every base part lies in one row-major tile, Prop. in Sec. 2.1).
"""

from __future__ import annotations

from dataclasses import dataclass

from . import encode, extract_i, extract_j


@dataclass(frozen=True)
class Part:
    """A sub-matrix (M, sigma, r, c) with its Cartesian start (i0, j0)."""
    sigma: int
    r: int
    c: int
    i0: int
    j0: int


@dataclass(frozen=True)
class Leaf:
    """One base-case multiplication S_A += S_B * S_C on contained parts, with its
    local ranges (i, j, l) inside the top-level product."""
    A: Part
    B: Part
    C: Part
    i_lo: int
    i_hi: int
    j_lo: int
    j_hi: int
    l_lo: int
    l_hi: int


def _part(i0: int, j0: int, r: int, c: int, m: int, T: int) -> Part:
    sigma = encode(i0, j0, m, T) if (r > 0 and c > 0) else -1
    return Part(sigma, r, c, i0, j0)


def step2_split(alpha: int, lam: int, S: Part, m: int, T: int):
    """Step 2: the four parts S'_{NW,NE,SW,SE} of S inside the quadrants of the
    aligned block (alpha, lambda). Returns a list of 4 Parts (possibly empty)."""
    lam_q = lam // 4
    e_NE = alpha + 2 * lam_q - 1
    e_SW = alpha + 3 * lam_q - 1
    i_S = extract_i(S.sigma, m, T)
    j_S = extract_j(S.sigma, m, T)
    r_N = extract_i(e_NE, m, T) - i_S + 1
    c_W = extract_j(e_SW, m, T) - j_S + 1
    r_N = min(max(r_N, 0), S.r)
    c_W = min(max(c_W, 0), S.c)
    r_Sth = S.r - r_N
    c_E = S.c - c_W
    return [
        _part(i_S, j_S, r_N, c_W, m, T),                # NW
        _part(i_S, j_S + c_W, r_N, c_E, m, T),          # NE
        _part(i_S + r_N, j_S, r_Sth, c_W, m, T),        # SW
        _part(i_S + r_N, j_S + c_W, r_Sth, c_E, m, T),  # SE
    ]


class Recursion:
    """Runs the recursion for S_A += S_B * S_C.

    Top level: S_A is (i_A, j_A, M, N) in A, S_B is (i_B, j_B, M, K) in B and
    S_C is (i_C, j_C, K, N) in C, all matrices (2^m T')^2 Morton-hybrid.
    """

    def __init__(self, m: int, T: int, sA, sB, sC):
        self.m, self.T = m, T
        (self.iA, self.jA, self.M, self.N) = sA
        (self.iB, self.jB, M2, self.K) = sB
        (self.iC, self.jC, K2, N2) = sC
        if (M2, K2, N2) != (self.M, self.K, self.N):
            raise ValueError("incompatible sub-matrix shapes")
        self.leaves: list[Leaf] = []
        self.calls = 0                 # recursive MM calls made (all levels)
        self.max_children = 0          # most compatible combinations at one level

    # local index ranges restricted by a part of each matrix
    def _ranges_A(self, P: Part):
        return (P.i0 - self.iA, P.i0 - self.iA + P.r), (P.j0 - self.jA, P.j0 - self.jA + P.c)

    def _ranges_B(self, P: Part):
        return (P.i0 - self.iB, P.i0 - self.iB + P.r), (P.j0 - self.jB, P.j0 - self.jB + P.c)

    def _ranges_C(self, P: Part):
        return (P.i0 - self.iC, P.i0 - self.iC + P.r), (P.j0 - self.jC, P.j0 - self.jC + P.c)

    def run(self):
        n = (1 << self.m) * self.T
        lam = n * n
        m, T = self.m, self.T
        if self.M == 0 or self.N == 0 or self.K == 0:
            return self.leaves
        SA = _part(self.iA, self.jA, self.M, self.N, m, T)
        SB = _part(self.iB, self.jB, self.M, self.K, m, T)
        SC = _part(self.iC, self.jC, self.K, self.N, m, T)
        self._mm(0, lam, SA, 0, lam, SB, 0, lam, SC)
        return self.leaves

    def _mm(self, aA, lA, SA, aB, lB, SB, aC, lC, SC):
        self.calls += 1
        T = self.T
        if lA == T * T:
            (i_lo, i_hi), (j_lo, j_hi) = self._ranges_A(SA)
            (_, _), (l_lo, l_hi) = self._ranges_B(SB)
            self.leaves.append(Leaf(SA, SB, SC, i_lo, i_hi, j_lo, j_hi, l_lo, l_hi))
            return
        # Step 1: quadrants of each aligned block
        lq = lA // 4
        alphas_A = [aA + q * lq for q in range(4)]
        alphas_B = [aB + q * (lB // 4) for q in range(4)]
        alphas_C = [aC + q * (lC // 4) for q in range(4)]
        # Step 2: the part of S inside each quadrant
        PA = step2_split(aA, lA, SA, self.m, T)
        PB = step2_split(aB, lB, SB, self.m, T)
        PC = step2_split(aC, lC, SC, self.m, T)
        # Step 3: all combinations of quadrants; Step 4: compatible parts
        children = 0
        for t in range(4):
            if PA[t].r == 0 or PA[t].c == 0:
                continue
            (ia, ja) = self._ranges_A(PA[t])
            for u in range(4):
                if PB[u].r == 0 or PB[u].c == 0:
                    continue
                (ib, lb) = self._ranges_B(PB[u])
                for v in range(4):
                    if PC[v].r == 0 or PC[v].c == 0:
                        continue
                    (lc, jc) = self._ranges_C(PC[v])
                    i_lo, i_hi = max(ia[0], ib[0]), min(ia[1], ib[1])
                    j_lo, j_hi = max(ja[0], jc[0]), min(ja[1], jc[1])
                    l_lo, l_hi = max(lb[0], lc[0]), min(lb[1], lc[1])
                    if i_lo >= i_hi or j_lo >= j_hi or l_lo >= l_hi:
                        continue
                    m, T = self.m, self.T
                    cA = _part(self.iA + i_lo, self.jA + j_lo, i_hi - i_lo, j_hi - j_lo, m, T)
                    cB = _part(self.iB + i_lo, self.jB + l_lo, i_hi - i_lo, l_hi - l_lo, m, T)
                    cC = _part(self.iC + l_lo, self.jC + j_lo, l_hi - l_lo, j_hi - j_lo, m, T)
                    children += 1
                    self._mm(alphas_A[t], lq, cA, alphas_B[u], lB // 4, cB,
                             alphas_C[v], lC // 4, cC)
        self.max_children = max(self.max_children, children)


def leaves(m: int, T: int, sA, sB, sC):
    """Base-case triples of the recursion for S_A += S_B * S_C (see Recursion)."""
    return Recursion(m, T, sA, sB, sC).run()


def default_calls(T: int, M: int, N: int, K: int) -> int:
    """Base-case calls of the default recursive MM that divides the sub-matrices
    themselves (Sec. 2.2, first paragraph; the comparison of Table 1): each
    dimension above T' is halved (ceil / floor) and all 8 sub-products recurse;
    a product whose three dimensions are all <= T' is one base-case call.
    The paper does not print this algorithm; this is the standard divide-and-
    conquer MM on the sub-matrices' own dimensions (parity unpinned)."""
    if M == 0 or N == 0 or K == 0:
        return 0
    if M <= T and N <= T and K <= T:
        return 1

    def halves(x):
        return [x] if x <= T else [(x + 1) // 2, x // 2]

    return sum(default_calls(T, a, b, c) for a in halves(M) for b in halves(N) for c in halves(K))
