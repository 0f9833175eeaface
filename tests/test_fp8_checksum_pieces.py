"""The FP8 checksum operand holds B e exactly (reading R8), checked on the CPU.

The encode writes B e, a binary32 sum of at most 248 E4M3 values, as eight E4M3 pieces with
fixed scales 2^(9 - 4p): piece p is the nearest-even, saturating E4M3 value of r / 2^(9 - 4p),
r being what the previous pieces leave, and a piece below the smallest normal is flushed to
zero with its value carried. This restates that procedure from the E4M3 definition (OCP 8-bit
floating point: bias 7, 3 mantissa bits, subnormals at exponent field 0, no infinities) and
checks, on random sums and on random values of the grid such sums live on, that every
subtraction is exact, that nothing remains after eight pieces, and that the pieces'
magnitudes sum to at most 1.25 |B e| (the bound the threshold uses).
"""
import numpy as np


def e4m3_values():
    vals = set()
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue  # NaN
        v = (m / 8) * 2.0 ** -6 if e == 0 else (1 + m / 8) * 2.0 ** (e - 7)
        vals.add(-v if s else v)
    return np.array(sorted(vals))


GRID = e4m3_values()


def even_code(v):
    a = abs(v)
    if a == 0:
        return True
    e = int(np.floor(np.log2(a)))
    if e < -6:
        return int(round(a / 2.0 ** -9)) % 2 == 0
    return int(round((a / 2.0 ** e - 1) * 8)) % 2 == 0


def nearest_e4m3(x):
    if x >= 448:
        return 448.0
    if x <= -448:
        return -448.0
    i = int(np.searchsorted(GRID, x))
    lo, hi = GRID[max(i - 1, 0)], GRID[min(i, len(GRID) - 1)]
    if abs(x - lo) != abs(hi - x):
        return lo if abs(x - lo) < abs(hi - x) else hi
    return lo if even_code(lo) else hi


def pieces(S, n=8):
    r = np.float32(S)
    out = []
    for p in range(n):
        scale = 2.0 ** (9 - 4 * p)
        q = nearest_e4m3(float(np.float32(r * np.float32(1.0 / scale))))
        if abs(q) < 2.0 ** -6:
            q = 0.0
        piece = np.float32(q * scale)
        nxt = np.float32(r - piece)
        assert float(nxt) == float(r) - float(piece)  # exact in binary32
        r = nxt
        out.append(float(piece))
    return out, float(r)


def check(S):
    ps, rem = pieces(S)
    assert rem == 0.0, S
    if S != 0:
        assert sum(abs(p) for p in ps) <= 1.25 * abs(float(S)), S


def test_random_sums_of_e4m3_values():
    rng = np.random.default_rng(7)
    small, large = GRID[np.abs(GRID) < 2.0 ** -4], GRID[np.abs(GRID) > 100]
    for t in range(3000):
        L = int(rng.integers(1, 249))
        pool = (GRID, small, large)[t % 3]
        S = np.float32(0)
        for x in rng.choice(pool, L):
            S = np.float32(S + np.float32(x))
        check(S)


def test_values_of_the_grid_sums_live_on():
    # a binary32 sum of E4M3 values: a multiple of 2^-9 below 2^14, any binary32 value above
    rng = np.random.default_rng(8)
    for t in range(6000):
        if t % 2 == 0:
            S = np.float32(int(rng.integers(1, 2 ** 23)) * 2.0 ** -9)
        else:
            S = np.float32((1 + int(rng.integers(0, 2 ** 23)) / 2 ** 23) * 2.0 ** int(rng.integers(14, 17)))
        if abs(float(S)) < 248 * 448:
            check(S if t % 4 < 2 else -S)


def test_extremes():
    for S in (2.0 ** -9, -2.0 ** -9, 448.0 * 248, -448.0 * 248, 2.0 ** 14 - 2.0 ** -9, 2.0 ** 14 + 2.0 ** -9 * 4,
              float(np.nextafter(np.float32(2.0 ** 16), np.float32(0)))):
        if abs(S) <= 248 * 448:
            check(np.float32(S))
