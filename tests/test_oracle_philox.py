"""Pin the oracle's Philox-4x32-10 to the published known-answer vectors."""

import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        v = [int(x, 16) for x in line.split()]
        rows.append((v[0:4], v[4:6], v[6:10]))
    return rows


def test_known_answers(orc):
    rows = kat_rows()
    assert len(rows) == 3
    for ctr, key, out in rows:
        assert orc.philox4x32_10(ctr, key) == out


def test_counter_sensitivity(orc):
    """Changing any single counter or key bit changes the block (sanity)."""
    base = orc.philox4x32_10([1, 2, 3, 4], [5, 6])
    for w in range(4):
        c = [1, 2, 3, 4]
        c[w] ^= 1
        assert orc.philox4x32_10(c, [5, 6]) != base
    assert orc.philox4x32_10([1, 2, 3, 4], [5, 7]) != base
