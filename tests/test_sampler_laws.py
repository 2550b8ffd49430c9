"""Section 4's samplers as read here, pinned on exact rationals: DPRS
(Alg. 3) and ZPRS (Alg. 4) with k threads select element e with probability
w_e / sum(w) (the paper's correctness propositions).  Each element fires
independently with the probability its step of the algorithm computes, and the
returned index is the last firing one in the algorithm's order (sequence order
for DPRS; thread-major, the zig-zag order, for ZPRS), so the law is
p_e * prod over later elements of (1 - p).  A plausible misreading, e.g. an
inclusive instead of exclusive prefix in ZPRS, or sequence instead of
thread-major order, breaks the equality."""

from fractions import Fraction

import pytest


def _last_firing_law(order, p):
    law = {}
    for i, e in enumerate(order):
        q = p[e]
        for e2 in order[i + 1:]:
            q *= 1 - p[e2]
        law[e] = q
    return law


def dprs_law(w, k):
    n = len(w)
    p = {}
    wB = Fraction(0)
    iters = (n + k - 1) // k
    for i in range(iters):
        WL = [Fraction(w[j + i * k]) if j + i * k < n else Fraction(0) for j in range(k)]
        WP = [sum(WL[:j + 1], Fraction(0)) for j in range(k)]   # inclusive prefix in the iteration
        for j in range(k):
            e = j + i * k
            if e < n:
                p[e] = WL[j] / (WP[j] + wB) if WL[j] > 0 else Fraction(0)
        wB += WP[k - 1]
    return _last_firing_law(list(range(n)), p)


def zprs_law(w, k, inclusive=False, order="zigzag"):
    n = len(w)
    WL = [sum((Fraction(w[e]) for e in range(j, n, k)), Fraction(0)) for j in range(k)]
    WP = [sum(WL[:j + (1 if inclusive else 0)], Fraction(0)) for j in range(k)]   # exclusive prefix
    p = {}
    for j in range(k):
        P = WP[j]
        for e in range(j, n, k):
            P += w[e]
            p[e] = Fraction(w[e]) / P if w[e] > 0 else Fraction(0)
    seq = [e for j in range(k) for e in range(j, n, k)] if order == "zigzag" else list(range(n))
    return _last_firing_law(seq, p)


CASES = [
    ([3], 2),
    ([1, 2, 3, 4, 5, 6], 3),        # the size of the paper's running example (n = 6, k = 3)
    ([5, 1, 0, 2, 7, 1, 1, 3], 3),  # a zero weight
    ([1, 1, 1, 1, 1, 1, 1], 4),
    ([2, 9, 4, 0, 0, 6, 1, 8, 3, 5, 2], 4),
    ([1, 3, 2, 5], 8),              # more threads than elements
]


@pytest.mark.parametrize("w,k", CASES)
def test_dprs_law(w, k):
    law = dprs_law(w, k)
    tot = sum(w)
    for e, x in enumerate(w):
        assert law[e] == Fraction(x, tot)


@pytest.mark.parametrize("w,k", CASES)
def test_zprs_law(w, k):
    law = zprs_law(w, k)
    tot = sum(w)
    for e, x in enumerate(w):
        assert law[e] == Fraction(x, tot)


def test_zprs_misreadings_fail():
    w, k = [2, 9, 4, 0, 0, 6, 1, 8, 3, 5, 2], 4
    tot = sum(w)
    exact = [Fraction(x, tot) for x in w]
    assert [zprs_law(w, k, inclusive=True)[e] for e in range(len(w))] != exact
    assert [zprs_law(w, k, order="sequence")[e] for e in range(len(w))] != exact
